"""Structure checks and canonical forms for head/next fragment lists.

List order inside a pixel or octant depends on the order in which concurrent
insertions reach the head (Section 3.1: fragments are kept in the order the
rasteriser produced them), so two correct implementations can link the same
records differently. These helpers validate the structure of a list set and
reduce it to a canonical, order-free form: the sorted multiset of
(slot, record) pairs.
"""
import numpy as np


def list_owner(head: np.ndarray, nxt: np.ndarray, n: int) -> np.ndarray:
    """Slot owning each stored record 0..n-1, asserting a valid list set.

    Valid means: heads and next entries are -1 or in [0, n); no record is the
    head of two slots or the successor of two records; every record is reached
    from exactly one head; no cycles.
    """
    head = np.asarray(head).astype(np.int64)
    nxt = np.asarray(nxt[:n]).astype(np.int64)
    assert ((head == -1) | ((head >= 0) & (head < n))).all(), "head out of range"
    assert ((nxt == -1) | ((nxt >= 0) & (nxt < n))).all(), "next out of range"
    slots = np.nonzero(head >= 0)[0]
    hv = head[slots]
    assert np.unique(hv).size == hv.size, "record heads two lists"
    succ = nxt[nxt >= 0]
    assert np.unique(succ).size == succ.size, "record follows two records"
    assert np.intersect1d(hv, succ).size == 0, "head record also has a predecessor"
    assert hv.size + succ.size == n, "records unreachable from any head"
    # predecessor pointers; heads point to themselves
    anc = np.arange(n, dtype=np.int64)
    src = np.nonzero(nxt >= 0)[0]
    anc[nxt[src]] = src
    is_head = np.zeros(n, bool)
    is_head[hv] = True
    for _ in range(int(np.ceil(np.log2(max(n, 2)))) + 2):
        if is_head[anc].all():
            break
        anc = anc[anc]
    assert is_head[anc].all(), "cycle in lists"
    owner_of_head = np.full(n, -1, np.int64)
    owner_of_head[hv] = slots
    return owner_of_head[anc]


def list_lengths(head, nxt, n, n_slots=None):
    owner = list_owner(head, nxt, n)
    return np.bincount(owner, minlength=n_slots or len(head))


def canonical(owner: np.ndarray, records: np.ndarray) -> np.ndarray:
    """Sorted (slot, key, tri, nrm) rows: the order-free content of a list set."""
    rows = np.empty(owner.size, dtype=[("slot", "<i8"), ("key", "<u8"), ("tri", "<u4"), ("nrm", "<u4")])
    rows["slot"] = owner
    rows["key"] = records["key"][: owner.size]
    rows["tri"] = records["tri"][: owner.size]
    rows["nrm"] = records["nrm"][: owner.size]
    return np.sort(rows, order=["slot", "key", "tri", "nrm"])


def walk(head, nxt, slot):
    """Indices of one list from head to end."""
    out = []
    i = int(head[slot])
    while i != -1:
        out.append(i)
        i = int(nxt[i])
        assert len(out) <= nxt.size
    return out
