"""Element-by-element comparison of a GPU build's host copy with the oracle's
output (serialWT, Fig. 1).  Integer output: zero tolerance."""
import numpy as np


def node_levels(nid: np.ndarray) -> np.ndarray:
    """Level of every heap id (root 0 on level 0; children 2id+1, 2id+2)."""
    nid = nid.astype(np.int64)
    lev = np.floor(np.log2(nid + 1)).astype(np.int64)
    lev -= ((np.int64(1) << lev) - 1 > nid).astype(np.int64)   # float rounding guards
    lev += ((np.int64(1) << (lev + 1)) - 1 <= nid).astype(np.int64)
    return lev


def check_nodes(E: np.ndarray, ref: dict) -> None:
    """The oracle's node table (heap id, bitmap offset and length of every
    non-empty node) read back from the node starts E of a GPU build: node p of
    level l starts at E[p << (L-l)] and ends at E[(p+1) << (L-l)]."""
    L = ref["L"]
    nid = ref["node_id"].astype(np.int64)
    if nid.size == 0:
        return
    lev = node_levels(nid)
    p = nid - ((np.int64(1) << lev) - 1)
    E = E.astype(np.int64)
    lo = E[p << (L - lev)]
    hi = E[(p + 1) << (L - lev)]
    assert np.array_equal(lo, ref["node_start"].astype(np.int64))
    assert np.array_equal(hi - lo, ref["node_len"].astype(np.int64))


def compare_with_oracle(out: dict, ref: dict) -> None:
    """Bitmaps (padding bits included), directories, zero counts, node table."""
    assert out["status"] == 0
    assert np.array_equal(out["bits"], ref["bits"])
    assert np.array_equal(out["rank"], ref["rank"])
    assert np.array_equal(out["zeros"], ref["zeros"])
    check_nodes(out["node_start"], ref)
