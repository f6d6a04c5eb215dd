"""Shared helpers of the test suite (comparison of decision dictionaries)."""
import numpy as np

FIELDS = ("mvx", "mvy", "sad", "satd", "cost", "best", "split", "evaluated")
LEAF_FIELDS = ("leaf_depth", "leaf_mvx", "leaf_mvy")


def ctu_cu_mask(dims, ctu, ctu_mask):
    """Per-depth boolean masks of the CUs that lie in sampled CTUs."""
    cc, cr = dims[0]
    m = np.asarray(ctu_mask, dtype=bool).reshape(cr, cc)
    out = []
    for d, (c, r) in enumerate(dims):
        k = 1 << d
        rows = np.arange(r) // k
        cols = np.arange(c) // k
        out.append(m[np.ix_(rows, cols)].reshape(-1))
    return out


def assert_decisions_equal(gpu, ora, ctu=64, ctu_mask=None, where=""):
    """Bit-exact comparison of every decision array (optionally only inside
    the sampled CTUs)."""
    assert gpu["grid"] == ora["grid"], where
    dims = gpu["grid"]
    masks = ctu_cu_mask(dims, ctu, ctu_mask) if ctu_mask is not None else None
    for k in FIELDS:
        for d in range(len(dims)):
            g, o = np.asarray(gpu[k][d]), np.asarray(ora[k][d])
            if masks is not None:
                g, o = g[masks[d]], o[masks[d]]
            if not np.array_equal(g, o):
                bad = np.flatnonzero(g != o)
                raise AssertionError(f"{where}: field {k} depth {d}: {bad.size} mismatches, first at "
                                     f"{bad[:5].tolist()} gpu={g[bad[:5]].tolist()} oracle={o[bad[:5]].tolist()}")
    c8, r8 = gpu["grid8"]
    m8 = None
    if ctu_mask is not None:
        cc, cr = dims[0]
        k = ctu // 8
        mm = np.asarray(ctu_mask, dtype=bool).reshape(cr, cc)
        m8 = mm[np.ix_(np.arange(r8) // k, np.arange(c8) // k)].reshape(-1)
    for k in LEAF_FIELDS:
        g, o = np.asarray(gpu[k]), np.asarray(ora[k])
        if m8 is not None:
            g, o = g[m8], o[m8]
        if not np.array_equal(g, o):
            bad = np.flatnonzero(g != o)
            raise AssertionError(f"{where}: {k}: {bad.size} mismatches at {bad[:5].tolist()}")


def dep_from(out, size, **kw):
    d = {"ref_size": size, "leaf_depth": out["leaf_depth"], "leaf_mvx": out["leaf_mvx"],
         "leaf_mvy": out["leaf_mvy"]}
    d.update(kw)
    return d
