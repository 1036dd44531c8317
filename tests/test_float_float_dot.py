"""The float-float dot product that the FP32 path's ghost kernel uses for the six
projections, checked on the CPU against exact rational sums.

Each FP64 weight w is stored as hi = fl32(w), lo = fl32(w - hi); a term hi*q
(q an FP32 field value) is split exactly into p + e with p = fl32(hi*q) and
e = fma(hi, q, -p); fl32(lo*q + e) is the term's low part; p enters the running
sum through Knuth's two-sum and every rounding error goes to the low word; two
lanes sum alternate entries and are combined the same way; the two words are
added in FP64 at the end.  This is the compensated dot product "Dot2" of
Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26, 2005, Sec. 5), whose error is
at most u|x.y| + gamma_n^2 sum|x_i y_i| for n terms, u = 2^-24, gamma_n =
n u / (1 - n u); the weight split adds at most 2^-48 sum|w q|.  Below, IEEE
float32 arithmetic (numpy) stands in for the kernel's FP32 instructions; the
weight rows are the oracle's cloud rows (and their combinations) of a cylinder
case, and the field values include sums with heavy cancellation, where plain
FP32 sums fail the same bound by orders of magnitude."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2609_24785_b300 import workloads
from _helpers import make_oracle

F32 = np.float32
U = 2.0 ** -24


def _split(w):
    hi = F32(w)
    return hi, F32(float(w) - float(hi))


def _two_sum_acc(hi, lo, p, e):
    t = F32(hi + p)
    bp = F32(t - hi)
    err = F32(F32(hi - F32(t - bp)) + F32(p - bp))
    return t, F32(lo + F32(err + e))


def _term(w, q):
    """(p, e) of one term: p = fl32(hi q), e = fl32(lo q + (hi q - p))."""
    hi, lo = _split(w)
    p = F32(hi * q)
    e = F32(float(hi) * float(q) - float(p))           # exact: hi q - p fits an FP32 number
    e = F32(float(lo) * float(q) + float(e))           # the FMA with the low weight (one rounding)
    return p, e


def dot2(w, q, lanes=2):
    """The kernel's arithmetic: `lanes` partial float-float sums over alternate
    entries, combined pairwise, returned as an FP64 number."""
    parts = []
    for lane in range(lanes):
        hi, lo = F32(0), F32(0)
        for j in range(lane, len(w), lanes):
            p, e = _term(w[j], q[j])
            hi, lo = _two_sum_acc(hi, lo, p, e)
        parts.append((hi, lo))
    hi, lo = parts[0]
    for h2, l2 in parts[1:]:
        hi, lo = _two_sum_acc(hi, lo, h2, l2)
    return float(hi) + float(lo)


def naive_f32(w, q):
    s = F32(0)
    for wj, qj in zip(w, q):
        s = F32(s + F32(F32(wj) * qj))
    return float(s)


def exact(w, q):
    return sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(w, q))


def _bound(w, q):
    """(gamma_n^2 + 2^-47) sum|w q| + 2^-52 |w.q|: Dot2's bound with the final
    rounding to FP32 replaced by the FP64 addition of the two words, plus the
    weight split."""
    n = len(w)
    g = n * U / (1 - n * U)
    absum = float(sum(abs(Fraction(float(a)) * Fraction(float(b))) for a, b in zip(w, q)))
    return (g * g + 2.0 ** -47) * absum + 2.0 ** -52 * abs(float(exact(w, q))), absum


def _weight_rows(max_rows=120):
    case = workloads.cylinder_pulse(256)
    o = make_oracle(case)
    rows = []
    for g in range(min(o.n_ghost, max_rows // 3)):
        G = o.ghost(g)
        L = G["L"]
        rows.append(L[0])                               # interpolation to the boundary point
        rows.append(G["c"] @ L)                         # the combinations used by the ghost fill
        rows.append(G["ct"] @ L)
    return [np.asarray(r, dtype=np.float64) for r in rows if len(r) > 1]


def test_weight_rows_cover_real_clouds():
    rows = _weight_rows()
    sizes = [len(r) for r in rows]
    assert len(rows) >= 60 and min(sizes) >= 6 and max(sizes) <= 120


@pytest.mark.parametrize("kind", ["random", "offset_cancel"])
def test_dot2_error_within_bound(kind):
    rng = np.random.Generator(np.random.PCG64(2609))
    worst_ff, worst_naive = 0.0, 0.0
    naive_fails = 0
    for w in _weight_rows():
        if kind == "random":
            q = rng.uniform(-1, 1, len(w)).astype(F32)
        else:
            # zero-sum weights against values 1000 + O(1): the result is
            # O(|w|) while sum |w q| is O(1000 |w|)
            w = w - w.mean()
            q = (1000.0 + rng.uniform(-1, 1, len(w))).astype(F32)
        ex = exact(w, q)
        bnd, absum = _bound(w, q)
        e_ff = abs(Fraction(dot2(w, q)) - ex)
        e_nv = abs(Fraction(naive_f32(w, q)) - ex)
        assert float(e_ff) <= bnd, (len(w), float(e_ff), bnd)
        worst_ff = max(worst_ff, float(e_ff) / absum)
        worst_naive = max(worst_naive, float(e_nv) / absum)
        naive_fails += float(e_nv) > bnd
    print("%s: worst |err| / sum|w q|: float-float %.2e, plain FP32 %.2e" % (kind, worst_ff, worst_naive))
    # the check discriminates: plain FP32 sums break the same bound
    assert naive_fails > 0 and worst_naive > 1e3 * max(worst_ff, 2.0 ** -60)


def test_dot2_single_lane_and_lane_combine_agree_closely():
    """The lane split changes only the order of the compensated sums."""
    rng = np.random.Generator(np.random.PCG64(7))
    for w in _weight_rows(30):
        q = rng.uniform(-1, 1, len(w)).astype(F32)
        a, b = dot2(w, q, lanes=1), dot2(w, q, lanes=2)
        _, absum = _bound(w, q)
        assert abs(a - b) <= 2 * (len(w) * U) ** 2 * absum + 2.0 ** -46 * absum
