"""Parity at full UHD size: a 3840x2160 10-bit source pair and its six rungs
2160p / 1440p / 1080p / 720p / 540p / 360p, the 360p rung analysed
independently at +-64 and the other rungs as dependents at +-8 with the
depth window n, n+1 (inter-resolution reuse with refinement, Sec. 4.3 and
Sec. 6.3), QPs from {22, 27, 32, 37}.  The analyses run in the launch
configuration the bench times: a batch of ladder frames captured into a
CUDA graph and replayed.

The oracle analyses the 360p reference rung in full (every CU of every
depth); dependent rungs and the +-64 independent searches of the large
rungs are compared on seeded CTU samples that always hold the ragged
bottom-right CTU (the oracle computes sampled CTUs one by one).  The
cascaded chain of the proposed multi-encoding scheme (Sec. 6.5) is checked
the same way, each tier against the oracle's analysis of its parent."""
import numpy as np
import pytest

import oracle
from paper_2301_12191_gb300 import synth
from helpers import assert_decisions_equal, dep_from

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2301_12191_gb300 import ladder as L  # noqa: E402

SOURCE = (3840, 2160)
RUNGS = [(3840, 2160), (2560, 1440), (1920, 1080), (1280, 720), (960, 540), (640, 360)]
REF = 5
R, RR = 64, 8
QPS = [22, 27, 32, 37]
CHAIN = [2, 3, 4, 5, 5, -1]   # 360 -> 720 -> 1440 and 360 -> 540 -> 1080 -> 2160


def _sequence(seed):
    """Two consecutive frames of one seeded 2160p 10-bit ladder sequence (the
    bench's recipe: texture amplitude x4, noise sigma 8, global motion up to
    +-8 and patch motion up to +-12 at 416 wide, scaled by 3840 / 416)."""
    W = SOURCE[0]
    return synth.ladder_sequence(seed, 2, source=SOURCE, rungs=RUNGS, bit_depth=10,
                                 global_range=8 * W // 416, patch_range=12 * W // 416,
                                 patch_size=int(round(64 * W / 416 / 8)) * 8, noise_sigma=8)


def _planes(seq):
    """Per rung (cur, ref) = (frame 1, frame 0) as device planes, plus the host planes."""
    host = [(seq[1][r], seq[0][r]) for r in range(len(RUNGS))]
    return [(L.device_plane(c), L.device_plane(f)) for c, f in host], host


def _sample(w, h, k, seed):
    dims, _ = oracle.grid(w, h, 64)
    n = dims[0][0] * dims[0][1]
    mask = np.zeros(n, dtype=np.uint8)
    mask[np.random.default_rng(seed).choice(n, size=min(n, k), replace=False)] = 1
    mask[-1] = 1   # the ragged bottom-right CTU
    return mask


def test_uhd_ladder_graph_batch():
    """Two ladder frames (QP 22 and 27) in one captured batch, replayed twice."""
    seqs = [_sequence(3000 + l) for l in range(2)]
    qps = [QPS[l % len(QPS)] for l in range(2)]
    with L.Ladder(RUNGS, REF, bit_depth=10, ctu_size=64, search_range=R, refine_range=RR, max_frames=2) as lad:
        dev, host = zip(*[_planes(s) for s in seqs])
        items = [(k, qps[k], list(dev[k])) for k in range(2)]
        stream = torch.cuda.Stream()
        graph = lad.capture_batch(items, stream)
        for _ in range(2):
            graph.launch(stream)
        stream.synchronize()
        got = [[lad.fetch(r, k) for r in range(len(RUNGS))] for k in range(2)]
        lad.sync()
        graph.close()
    for k in range(2):
        c, f = host[k][REF]
        ora_ref = oracle.analyze(c, f, qp=qps[k], search_range=R, ctu=64)
        assert_decisions_equal(got[k][REF], ora_ref, 64, where=f"frame {k} 360p reference")
        for r, (w, h) in enumerate(RUNGS):
            if r == REF:
                continue
            mask = _sample(w, h, 16, 100 * k + r)
            ora = oracle.analyze(*host[k][r], qp=qps[k], search_range=RR, ctu=64, ctu_mask=mask,
                                 dep=dep_from(ora_ref, RUNGS[REF]))
            assert_decisions_equal(got[k][r], ora, 64, ctu_mask=mask, where=f"frame {k} rung {w}x{h}")


def test_uhd_independent_baseline_sampled():
    """The per-rung baseline of the speedup: +-64 full search on every rung
    (batched independent analyses), sampled CTUs of each rung."""
    seq = _sequence(3002)
    qp = QPS[2]
    with L.Ladder(RUNGS, REF, bit_depth=10, ctu_size=64, search_range=R, refine_range=RR, max_frames=1) as lad:
        dev, host = _planes(seq)
        lad.analyze_batch_independent([(0, qp, dev)])
        got = [lad.fetch(r, 0) for r in range(len(RUNGS))]
    for r, (w, h) in enumerate(RUNGS):
        mask = _sample(w, h, 3, 50 + r)
        ora = oracle.analyze(*host[r], qp=qp, search_range=R, ctu=64, ctu_mask=mask)
        assert_decisions_equal(got[r], ora, 64, ctu_mask=mask, where=f"independent {w}x{h}")


def test_uhd_cascaded_chain():
    """360p -> 720p -> 1440p and 360p -> 540p -> 1080p -> 2160p, one frame:
    each dependent rung against the oracle's dependent analysis of its own
    parent's oracle decisions (parents in full, the top rungs sampled)."""
    seq = _sequence(3003)
    qp = QPS[3]
    with L.Ladder(RUNGS, REF, bit_depth=10, ctu_size=64, search_range=R, refine_range=RR, max_frames=1) as lad:
        lad.set_parents(CHAIN)
        dev, host = _planes(seq)
        lad.analyze_batch([(0, qp, dev)])
        got = [lad.fetch(r, 0) for r in range(len(RUNGS))]
    ora = {REF: oracle.analyze(*host[REF], qp=qp, search_range=R, ctu=64)}
    assert_decisions_equal(got[REF], ora[REF], 64, where="chain 360p reference")
    full = {3, 4, 2}              # parents of later tiers: compared in full
    for r in (3, 4, 2, 1, 0):     # parents before children
        p = CHAIN[r]
        w, h = RUNGS[r]
        mask = None if r in full else _sample(w, h, 16, 70 + r)
        ora[r] = oracle.analyze(*host[r], qp=qp, search_range=RR, ctu=64, ctu_mask=mask,
                                dep=dep_from(ora[p], RUNGS[p]))
        assert_decisions_equal(got[r], ora[r], 64, ctu_mask=mask, where=f"chain rung {w}x{h} (parent {RUNGS[p]})")
