"""The all-core CPU baseline runs the oracle's unchanged functions on
several threads; its results must be identical to the single-threaded
oracle's: the same records in the same order, the same visibility and
colours for every view."""
import numpy as np

from paper_2211_15460_gb300 import scenes


def test_threaded_oracle_identical_to_single_thread(oracle_mod):
    from oracle import threads

    w = scenes.workload_spheres_256()
    for mode, cam, pitch in ((oracle_mod.VIEW, w.capture, 0.0), (oracle_mod.NORMAL, None, w.normal_pitch),
                             (oracle_mod.AXIS3, None, w.normal_pitch)):
        one = oracle_mod.fragments(w.scene, mode, cam, pitch)[0]
        many = threads.fragments(w.scene, mode, cam, pitch, threads=5)
        assert many.dtype == one.dtype and np.array_equal(many, one)
    pofa = oracle_mod.pofa_sort(one)
    views = [scenes.orbit_camera(w.scene, 96, 64, orbit_deg=d) for d in (0.0, 30.0, 75.0)]
    got = threads.render_views(pofa, w.scene, views, w.lights, 1, threads=3)
    for v, (vis, rgba) in zip(views, got):
        vis1, rgba1 = oracle_mod.render(pofa, w.scene, v, w.lights, 1)
        assert np.array_equal(vis, vis1) and np.array_equal(rgba, rgba1)
