"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a scratch copy of the oracle's C source
(a wrong sign, index, rounding mode, operand order or bit position), builds
it, and runs the pin suite against it in a subprocess: the suite must fail.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fhv_oracle.c")

MUTATIONS = [
    ("top-left rule flipped", "return dy < 0 || (dy == 0 && dx < 0);", "return dy > 0 || (dy == 0 && dx < 0);"),
    ("position rounding floors", "(2 * num + A)", "(2 * num)"),
    ("barycentric weights rotated", "(__int128)w[k] * (__int128)t.Q[k][c]", "(__int128)w[k] * (__int128)t.Q[(k + 1) % 3][c]"),
    ("morton x bit moved", "<< (3 * k + 2);", "<< (3 * k);"),
    ("normal operands swapped", "float a1 = fw[1] * t.N[1][c];", "float a1 = fw[1] * t.N[2][c];"),
    ("octahedral fold sign", "if (nz < 0.0f) {", "if (nz > 0.0f) {"),
    ("bitangent handedness", "cross3f(nn, tt, bb);", "cross3f(tt, nn, bb);"),
    ("list link dropped", "c->next[n] = c->head[slot];", "c->next[n] = -1;"),
    ("occupancy bit index", "1u << (child & 7u);", "1u << (child & 3u);"),
    ("inclusive offsets", "off[base + o] = run;", "off[base + o] = run + cnt[base + o];"),
    ("splat anchor rounds", "float fx = floorf(sx - half)", "float fx = rintf(sx - half)"),
    ("depth code reversed", "float tz = (z - cam->z0) * qscale;", "float tz = (cam->z1 - z) * qscale;"),
    ("no back-facing clamp", "if (ndl < 0.0) ndl = 0.0;", ""),
    ("quantisation rounds", "float f = floorf(u);", "float f = rintf(u);"),
    ("vertex snap shifted", "out->X[v] = snap256(sx);", "out->X[v] = snap256(sx) + 1;"),
    ("snorm16 floors", "(int32_t)rintf(px * 32767.0f)", "(int32_t)floorf(px * 32767.0f)"),
    ("octant lower bound", "if (pre < o) lo = mid + 1; else hi = mid;", "if (pre <= o) lo = mid + 1; else hi = mid;"),
    ("ray transmittance not attenuated", "T *= 1.0 - a;", "T *= a;"),
    ("ray colour without transmittance", "C[c] += T * a * col[c];", "C[c] += a * col[c];"),
    ("ray hits back to front",
     "return x->pix < y->pix ? -1 : 1;\n    if (x->key != y->key) return x->key < y->key ? -1 : 1;",
     "return x->pix < y->pix ? -1 : 1;\n    if (x->key != y->key) return x->key > y->key ? -1 : 1;"),
    ("ray opacity from transmittance", "rgba[4 * p + 3] = (float)(1.0 - T);", "rgba[4 * p + 3] = (float)T;"),
]


@pytest.mark.slow
@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, "mutation site not unique"
    mutated = tmp_path / "fhv_oracle.c"
    mutated.write_text(text.replace(old, new))
    env = dict(os.environ, FHV_ORACLE_SRC=str(mutated))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x", "-q",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode != 0, f"pins did not catch: {name}\n{r.stdout[-2000:]}"
    shutil.rmtree(tmp_path / "_build", ignore_errors=True)


GAPFILL_SRC = os.path.join(ROOT, "oracle", "gapfill.py")
GAPFILL_MUTATIONS = [
    ("conv taps transposed", "xp[:, ky:ky + h, kx:kx + wd, :], w[:, ky, kx, :])",
     "xp[:, ky:ky + h, kx:kx + wd, :], w[:, kx, ky, :])"),
    ("weight gradient tap mirrored", 'dw[:, ky, kx, :] = np.einsum("nijo,nijc->oc", dy, xp[:, ky:ky + h, kx:kx + wd, :])',
     'dw[:, ky, kx, :] = np.einsum("nijo,nijc->oc", dy, xp[:, 2 - ky:2 - ky + h, kx:kx + wd, :])'),
    ("flip not transposed", ".transpose(3, 1, 2, 0))", ".transpose(0, 1, 2, 3))"),
    ("adam without bias correction", "mh = m / (1.0 - b1 ** step)", "mh = m"),
    ("loss gradient sign", "g[..., :3] = grad_scale * d", "g[..., :3] = -grad_scale * d"),
    ("loss ignores the base", "d = d + np.asarray(base, np.float64)[..., :3]", "d = d"),
    ("bf16 ties away from zero", "r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16", "r = ((u + 0x8000) >> 16) << 16"),
    ("octahedral fold flipped", "fold = z < 0", "fold = z > 0"),
    ("relu dropped", "y = np.maximum(y, 0.0)", "y = y"),
    ("feature normal axes swapped", "f[hit, 5] = n @ np.asarray(cam.right, np.float64)",
     "f[hit, 5] = n @ np.asarray(cam.up, np.float64)"),
    ("feature normal on the view direction", "f[hit, 6] = n @ np.asarray(cam.up, np.float64)",
     "f[hit, 6] = n @ np.asarray(cam.fwd, np.float64)"),
    ("feature depth code shifted", "f[hit, 3] = (vis[hit] >> np.uint64(40))", "f[hit, 3] = (vis[hit] >> np.uint64(41))"),
]


@pytest.mark.slow
@pytest.mark.parametrize("name,old,new", GAPFILL_MUTATIONS, ids=[m[0] for m in GAPFILL_MUTATIONS])
def test_gapfill_pins_catch_planted_mistake(tmp_path, name, old, new):
    text = open(GAPFILL_SRC).read()
    assert text.count(old) == 1, "mutation site not unique"
    mutated = tmp_path / "gapfill.py"
    mutated.write_text(text.replace(old, new))
    env = dict(os.environ, FHV_GAPFILL_ORACLE_SRC=str(mutated))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_gapfill.py"), "-x",
                        "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch: {name}\n{r.stdout[-2000:]}"
