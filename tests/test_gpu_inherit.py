"""Dependent CUs whose candidate SADs are the sums of their sub-CUs'
(LADDER_TUNE_DEP_INHERIT).  A CU searched in pieces whose four sub-CUs are
evaluated around its own centre (Sec. 4.3: every dependent CU is refined
around the scaled vector of its co-located reference CU; here the four
quarters share that vector) is not searched: the SAD of a candidate over the
CU is the sum of its SADs over the four quarters.  The decisions equal the
oracle's with the knob on and off, and the searches skip exactly the CUs the
rule names: the device's count of SAD-candidate evaluations equals the count
recomputed here from the oracle's rules and evaluated flags."""
import pytest

import oracle
from paper_2301_12191_gb300 import synth
from helpers import assert_decisions_equal, dep_from

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2301_12191_gb300 import ladder as L  # noqa: E402

CTU = 64
DMAX = 3


def expected_evals(size, ev, dep, r, piece, depth_hi):
    """(every evaluated CU, searched CUs, inherited CUs, searched CUs below
    an inherited parent and grandparent) from the oracle's evaluated flags
    and rules."""
    W, H = size
    W8, H8 = (W + 7) // 8 * 8, (H + 7) // 8 * 8
    k2 = (2 * r + 1) ** 2
    cols = [(W8 + (CTU >> d) - 1) // (CTU >> d) for d in range(DMAX + 1)]
    rules = {}

    def rule(d, x, y):
        if (d, x, y) not in rules:
            rules[(d, x, y)] = oracle.derive_rule(size, dict(dep, depth_hi=depth_hi), d, x * (CTU >> d),
                                                  y * (CTU >> d), CTU)
        return rules[(d, x, y)]

    def evaluated(d, x, y):
        return x < cols[d] and bool(ev[d][y * cols[d] + x])

    inherited = set()
    total = 0
    for d in range(DMAX + 1):
        S = CTU >> d
        for i in range(ev[d].size):
            if not ev[d][i]:
                continue
            total += (S // 8) ** 2 * k2
            x, y = i % cols[d], i // cols[d]
            if S > piece and d < DMAX:
                kids = [(2 * x + (q & 1), 2 * y + (q >> 1)) for q in range(4)]
                if all(evaluated(d + 1, kx, ky) and rule(d + 1, kx, ky)[:2] == rule(d, x, y)[:2] for kx, ky in kids):
                    inherited.add((d, x, y))
    searched = total - sum(((CTU >> d) // 8) ** 2 * k2 for (d, _, _) in inherited)
    chains = sum(1 for (d, x, y) in inherited if d >= 1 and (d - 1, x // 2, y // 2) in inherited)
    return total, searched, len(inherited), chains


@pytest.mark.parametrize("bd,r,piece,depth_hi,staged", [
    (8, 4, 16, 1, 1),
    (10, 8, 16, 1, 1),
    (10, 8, 32, 1, 1),
    (10, 8, 16, 2, 1),   # three depths evaluated: inherited parents of inherited CUs
    (8, 4, 16, 2, 0),    # the L1 form of the search
    (10, 8, 16, 2, 2),
])
def test_inherited_cus_are_summed_not_searched(bd, r, piece, depth_hi, staged):
    pairs, _ = synth.ladder_pairs(23, source=(1280, 720), rungs=[(960, 540), (640, 360)], bit_depth=bd)
    sizes = [(w, h) for (w, h, _, _) in pairs]
    ref_i, qp, R = 2, 27, 16
    o_ref = oracle.analyze(pairs[ref_i][2], pairs[ref_i][3], qp=qp, search_range=R)
    dep = dep_from(o_ref, sizes[ref_i])
    o_dep = {i: oracle.analyze(pairs[i][2], pairs[i][3], qp=qp, search_range=r, dep=dict(dep, depth_hi=depth_hi))
             for i in (0, 1)}
    with L.Ladder(sizes, ref_i, bit_depth=bd, search_range=R, refine_range=r, depth_hi=depth_hi,
                  max_frames=1) as lad:
        planes = [(L.device_plane(c), L.device_plane(f)) for (_, _, c, f) in pairs]
        lad.set_tuning(dep_range=piece, dep_staged=staged)
        counted = {}
        for inherit in (0, 1):
            lad.set_tuning(dep_inherit=inherit)
            lad.sync()
            lad.dependent_evals()
            lad.analyze_reference(0, *planes[ref_i], qp)
            lad.analyze_dependents(0, [(i, *planes[i]) for i in (0, 1)], qp)
            lad.sync()
            counted[inherit] = lad.dependent_evals()
            assert_decisions_equal(lad.fetch(ref_i, 0), o_ref, CTU, where=f"reference, inherit={inherit}")
            for i in (0, 1):
                assert_decisions_equal(lad.fetch(i, 0), o_dep[i], CTU, where=f"rung {i}, inherit={inherit}")
            lad.release_frame(0)
    total = searched = n_inh = chains = 0
    for i in (0, 1):
        t, s, n, c = expected_evals(sizes[i], o_dep[i]["evaluated"], dep, r, piece, depth_hi)
        total, searched, n_inh, chains = total + t, searched + s, n_inh + n, chains + c
    assert counted[0] == total
    assert counted[1] == searched
    assert n_inh > 0 and searched < total
    if depth_hi == 2 and piece == 16:
        assert chains > 0
