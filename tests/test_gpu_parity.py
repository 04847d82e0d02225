"""GPU parity of the CUDA hot path (through the C-ABI) against the FP64 CPU oracle.

Tolerances:
  * FP64 mode: every particle within 1e-12 relative for a_i, g_i and tau_i.
  * mixed mode: 99.9th percentile of the per-particle relative error <= 1e-6 for a_i and
    for the gradient term g_i; the time-steps, which only steer the slow/fast split, within
    2e-6 relative at the 99.9th percentile (FP32 pair body with about twenty roundings and
    the approximate MUFU functions, each a few 1e-7).
  * index work (partition) bit-exact; kick/drift bit-exact (same roundings as the oracle).
Inputs are seeded synthetic Plummer spheres (equal or Kroupa masses), sized to span several
shared-memory tiles with a ragged tail.
"""

import math

import numpy as np
import pytest

import oracle
from paper_2011_14984_gb300 import ics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2011_14984_gb300 import frost
    frost.load()


def F(*a, **k):
    from paper_2011_14984_gb300.frost import Frost
    return Frost(*a, **k)


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    if a.ndim == 1:
        return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-300)


def p999(e):
    return float(np.percentile(e, 99.9))


def oracle_g(m, x, A, B, eps2=0.0):
    """g from the oracle with the accelerations of the same pass (same-set or cross)."""
    A = np.asarray(A, dtype=np.int32)
    B = np.asarray(B, dtype=np.int32)
    aA = oracle.acc(m, x, A, B, eps2=eps2)
    aB = oracle.acc(m, x, B, A, eps2=eps2)
    return aA, oracle.grad(m, x, A, aA, B, aB, eps2=eps2)


def cpu(t):
    return t.detach().cpu().numpy()


# ---------------------------------------------------------------------------------------
# acceleration and gradient passes
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("eps_soft", [0.0, 1e-3])
def test_accel_gradient_full_set(precision, eps_soft):
    n = 5000  # 39 tiles of 128 with a ragged tail
    m, x, v = ics.plummer(n, 101, masses=ics.kroupa_masses(n, 101))
    f = F(m, x, v, precision=precision, eps_soft=eps_soft)
    eps = 0.01
    out = f.accel_gradient(None, None, eps_grad=eps)
    A = np.arange(n, dtype=np.int32)
    a_ref, g_ref = oracle_g(m, x, A, A, eps2=eps_soft ** 2)
    at_ref = a_ref + eps * eps / 48.0 * g_ref
    ea = rel(cpu(out["acc"]), a_ref)
    eg = rel(cpu(out["grad"]), g_ref)
    et = rel(cpu(out["acc_tilde"]), at_ref)
    if precision == "fp64":
        assert ea.max() < 1e-12 and eg.max() < 1e-12 and et.max() < 1e-12, (ea.max(), eg.max())
    else:
        assert p999(ea) < 1e-6 and p999(eg) < 1e-6 and p999(et) < 1e-6, (p999(ea), p999(eg))
        assert ea.max() < 1e-5 and eg.max() < 2e-5
    f.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_accel_gradient_cross_pass(precision):
    """Disjoint active/source lists: the inter-level passes of Eqs. force-newton-inter and
    force-gradient-inter-1/2 (a_j of the sources due to the active set)."""
    n = 3001
    m, x, v = ics.plummer(n, 7)
    rng = np.random.default_rng(3)
    perm = rng.permutation(n).astype(np.int32)
    S, Fl = np.sort(perm[:700]), perm[700:]  # Fl unsorted on purpose
    f = F(m, x, v, precision=precision)
    eps = 0.05
    out = f.accel_gradient(S, Fl, eps_grad=eps)
    a_ref, g_ref = oracle_g(m, x, S, Fl)
    ea, eg = rel(cpu(out["acc"]), a_ref), rel(cpu(out["grad"]), g_ref)
    if precision == "fp64":
        assert ea.max() < 1e-12 and eg.max() < 1e-12
    else:
        assert p999(ea) < 1e-6 and p999(eg) < 1e-6, (p999(ea), p999(eg))
    # the same set given in another order is the intra-set pass
    out2 = f.accel_gradient(S[::-1].copy(), S, eps_grad=eps)
    a2, g2 = oracle_g(m, x, S[::-1], S[::-1])
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert rel(cpu(out2["acc"]), a2).max() < tol
    f.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("na,nb,eps_soft", [(5000, 3001, 0.0), (700, 61, 0.0), (3001, 5000, 1e-3), (1, 257, 0.0)])
def test_accel_pairwise_each_pair_once(precision, na, nb, eps_soft):
    """frost_accel_pairwise (both lines of Eq. force-newton-inter, every S x F pair evaluated
    once): both lists' accelerations against the oracle's one-sided sums, lists of Kroupa-mass
    particles with ragged tiles, in either order of sizes (the longer list takes the register
    side), softened, and a single particle; FP64 within 1e-12, mixed p99.9 <= 1e-6 and max
    <= 1e-5.  The pair terms are exact negatives up to the two weightings, so the total force
    m_a a_a + m_b a_b vanishes to round-off."""
    n = na + nb
    m, x, v = ics.plummer(n, 60 + na % 13, masses=ics.kroupa_masses(n, 60 + na % 13))
    perm = np.random.default_rng(na + nb).permutation(n).astype(np.int32)
    A, B = perm[:na], perm[na:]
    f = F(m, x, v, precision=precision, eps_soft=eps_soft)
    aa, ab = f.accel_pairwise(A, B)
    f.close()
    aa, ab = cpu(aa), cpu(ab)
    ra = oracle.acc(m, x, A, B, eps2=eps_soft ** 2)
    rb = oracle.acc(m, x, B, A, eps2=eps_soft ** 2)
    ea, eb = rel(aa, ra), rel(ab, rb)
    if precision == "fp64":
        assert ea.max() < 1e-12 and eb.max() < 1e-12, (ea.max(), eb.max())
    else:
        for e in (ea, eb):
            assert p999(e) < 1e-6 and e.max() < 1e-5, (p999(e), e.max())
    tot = (m[A][:, None] * aa).sum(0) + (m[B][:, None] * ab).sum(0)
    scale = (m[A][:, None] * np.abs(aa)).sum() + (m[B][:, None] * np.abs(ab)).sum()
    assert np.all(np.abs(tot) < (1e-14 if precision == "fp64" else 1e-7) * scale), tot / scale


@pytest.mark.parametrize("n,cross", [(5000, False), (16384, False), (5000, True), (9000, True)])
def test_symmetric_wmax_prepass_is_bit_identical(n, cross):
    """The prepass of the Newtonian pass that feeds a gradient, max_j m_j / r^3, with each pair
    once (one set, or two disjoint lists at once: r^2 is symmetric bit for bit and the maximum
    does not depend on the order): frost_accel_gradient gives the same a, a~ and g, bit for
    bit, as with the one-sided prepasses (Kroupa masses, so the dominant terms and slots
    differ between particles)."""
    m, x, v = ics.plummer(n, 50 + n % 7, masses=ics.kroupa_masses(n, 50 + n % 7))
    if cross:
        perm = np.random.default_rng(n).permutation(n).astype(np.int32)
        A, B = np.sort(perm[: n // 3]), perm[n // 3:]
    else:
        A = B = None
    out = {}
    for sc in (1, -1):
        f = F(m, x, v, precision="mixed", sym_cross=sc)
        o = f.accel_gradient(A, B, eps_grad=2.0 ** -7)
        out[sc] = {k: cpu(t) for k, t in o.items()}
        f.close()
    for k in out[1]:
        assert np.array_equal(out[1][k], out[-1][k]), k


def _check_gradient_pairwise(m, x, A, B, out, eps, bar=1e-6, cap=None):
    """Both lists of frost_accel_gradient_pairwise against the oracle: a, g and
    a~ = a + eps^2/48 g per list (the mixed bar at the 99.9th percentile, cap on the maximum).
    A list with fewer than 1000 sources is held to the cap alone: its g_i are sums of a few
    dozen Kroupa-mass terms, a few of them dominant, more than the 8 double-float slots of a
    split (the one-sided passes give 1.6e-6 at the 99.9th percentile on 700 against 61)."""
    for side, P, Q in (("a", A, B), ("b", B, A)):
        a_ref, g_ref = oracle_g(m, x, P, Q)
        ea, eg = rel(cpu(out["acc_" + side]), a_ref), rel(cpu(out["grad_" + side]), g_ref)
        et = rel(cpu(out["acc_tilde_" + side]), a_ref + eps * eps / 48.0 * g_ref)
        if len(Q) >= 1000:
            assert p999(ea) < bar and p999(eg) < bar and p999(et) < bar, (side, p999(ea), p999(eg), p999(et))
        if cap is not None:
            assert ea.max() < cap and eg.max() < cap and et.max() < cap, (side, ea.max(), eg.max(), et.max())


@pytest.mark.parametrize("sym_cross", [1, -1])
@pytest.mark.parametrize("na,nb", [(5000, 3001), (3001, 5000), (700, 61), (1, 257), (2049, 1)])
def test_accel_gradient_pairwise_matches_oracle(sym_cross, na, nb):
    """The force-gradient kick of two disjoint lists (both lines of Eqs.
    force-gradient-inter-1/2): with each pair once for both lists (sym_cross = 1, the longer
    list on the register side, the other reduced in a fixed order) and with two one-sided
    passes per kind (-1), both lists within the mixed bar of the oracle; ragged sizes, a list of
    one, lists given unsorted."""
    n = na + nb
    m, x, v = ics.plummer(n, 31 + n % 5, masses=ics.kroupa_masses(n, 31 + n % 5))
    perm = np.random.default_rng(n).permutation(n).astype(np.int32)
    A, B = perm[:na], perm[na:]
    f = F(m, x, v, precision="mixed", sym_cross=sym_cross)
    out = f.accel_gradient_pairwise(A, B, eps_grad=0.05)
    st = f.stats()
    f.close()
    assert (st["grad_pairs_symmetric"] == na * nb) == (sym_cross == 1)
    _check_gradient_pairwise(m, x, A, B, out, 0.05, cap=1e-5)


def test_accel_gradient_pairwise_is_deterministic_and_fp64_exact():
    """Repeated symmetric calls give the same bits (fixed-order sums, no atomics in a sum); the
    FP64 mode (two one-sided passes per kind) is within 1e-12 of the oracle on both lists."""
    n = 6000
    m, x, v = ics.plummer(n, 44)
    perm = np.random.default_rng(4).permutation(n).astype(np.int32)
    A, B = np.sort(perm[:3500]), perm[3500:]
    f = F(m, x, v, precision="mixed", sym_cross=1)
    o1 = {k: cpu(t) for k, t in f.accel_gradient_pairwise(A, B, eps_grad=0.05).items()}
    o2 = {k: cpu(t) for k, t in f.accel_gradient_pairwise(A, B, eps_grad=0.05).items()}
    f.close()
    for k in o1:
        assert np.array_equal(o1[k], o2[k]), k
    f = F(m, x, v, precision="fp64")
    out = f.accel_gradient_pairwise(A, B, eps_grad=0.05)
    f.close()
    for side, P, Q in (("a", A, B), ("b", B, A)):
        a_ref, g_ref = oracle_g(m, x, P, Q)
        assert rel(cpu(out["acc_" + side]), a_ref).max() < 1e-12
        assert rel(cpu(out["grad_" + side]), g_ref).max() < 1e-12


def test_accel_gradient_pairwise_full_slots_and_hard_binaries():
    """The two cases that stress the dominant terms, symmetric on both lists: (1) the outskirts
    of a Plummer sphere against its 96 central particles, where every outskirt particle has more
    dominant candidates than its slots (register side) and every core particle has hundreds of
    dominant partners (reduced side, no slot limit); the core side nearly cancels its own pull,
    so it is held to the bound of a floating-point sum, 1e-7 of the sum of the terms' sizes;
    (2) Kroupa masses with 5% hard binaries split between the lists: the hot sources in
    double-float on both sides, the mixed bar at the 99.9th percentile and 1e-5 at most."""
    n = 2000
    m, x, v = ics.plummer(n, 23)
    r = np.linalg.norm(x, axis=1)
    order = np.argsort(r).astype(np.int32)
    B = np.sort(order[:96])
    A = np.sort(order[-640:])
    f = F(m, x, v, precision="mixed", sym_cross=1)
    out = f.accel_gradient_pairwise(A, B, eps_grad=0.05)
    f.close()
    a_ref, g_ref = oracle_g(m, x, A, B)
    assert p999(rel(cpu(out["acc_a"]), a_ref)) < 1e-6 and p999(rel(cpu(out["grad_a"]), g_ref)) < 1e-6
    b_ref, gb_ref = oracle_g(m, x, B, A)
    d = x[A][None, :, :] - x[B][:, None, :]
    ri = 1.0 / np.linalg.norm(d, axis=2)
    Sa = (m[A][None, :] * ri ** 2).sum(1)
    da = a_ref[None, :, :] - b_ref[:, None, :]
    tg = (m[A][None, :] * ri ** 3)[..., None] * (da - 3.0 * ((d * da).sum(2) * ri ** 2)[..., None] * d)
    Sg = 2.0 * np.linalg.norm(tg, axis=2).sum(1)
    assert np.all(np.linalg.norm(cpu(out["acc_b"]) - b_ref, axis=1) < 1e-7 * Sa)
    assert np.all(np.linalg.norm(cpu(out["grad_b"]) - gb_ref, axis=1) < 1e-7 * Sg)

    n = 8192
    m, x, v = ics.plummer_kroupa_binaries(n, 17)
    perm = np.random.default_rng(5).permutation(n).astype(np.int32)
    A, B = np.sort(perm[:2500]), perm[2500:]
    f = F(m, x, v, precision="mixed", sym_cross=1)
    out = f.accel_gradient_pairwise(A, B, eps_grad=1e-3)
    f.close()
    _check_gradient_pairwise(m, x, A, B, out, 1e-3, cap=1e-5)


def test_accel_pairwise_rejects_overlapping_lists():
    from paper_2011_14984_gb300 import frost as fr
    m, x, v = ics.plummer(100, 3)
    f = F(m, x, v)
    with pytest.raises(fr.FrostError) as e:
        f.accel_pairwise(np.arange(0, 60, dtype=np.int32), np.arange(50, 100, dtype=np.int32))
    assert e.value.code == fr.FROST_EINVAL
    f.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_accel_gradient_pairwise_edge_cases(precision):
    """Overlapping lists are rejected (FROST_EINVAL); an empty list gives zeros for the other
    list (no partner: a = a~ = g = 0); a list of one against the rest matches the oracle."""
    from paper_2011_14984_gb300 import frost as fr
    m, x, v = ics.plummer(300, 9)
    f = F(m, x, v, precision=precision, sym_cross=1)
    with pytest.raises(fr.FrostError) as e:
        f.accel_gradient_pairwise(np.arange(0, 160, dtype=np.int32), np.arange(150, 300, dtype=np.int32), eps_grad=0.05)
    assert e.value.code == fr.FROST_EINVAL
    out = f.accel_gradient_pairwise(np.arange(0, 300, dtype=np.int32), np.zeros(0, dtype=np.int32), eps_grad=0.05)
    for k in ("acc_a", "acc_tilde_a", "grad_a"):
        assert np.all(cpu(out[k]) == 0.0), k
    A, B = np.array([17], dtype=np.int32), np.delete(np.arange(300, dtype=np.int32), 17)
    out = f.accel_gradient_pairwise(A, B, eps_grad=0.05)
    f.close()
    tol = 1e-12 if precision == "fp64" else 1e-5
    for side, P, Q in (("a", A, B), ("b", B, A)):
        a_ref, g_ref = oracle_g(m, x, P, Q)
        assert rel(cpu(out["acc_" + side]), a_ref).max() < tol
        assert rel(cpu(out["grad_" + side]), g_ref).max() < tol


def test_accel_gradient_cross_pass_full_slots():
    """A cross pass in which every deferred slot fills: 640 particles of the outskirts of a
    Plummer sphere against the 96 particles nearest its centre.  Seen from afar the core's
    terms are all within a factor 16 of the largest, so each particle has more candidates than
    its 8 double-float slots in every j-split (the rest stay in the FP32 sums), and the
    one-warp kernels share several rounds of deferred terms per warp."""
    n = 2000
    m, x, v = ics.plummer(n, 23)
    r = np.linalg.norm(x, axis=1)
    order = np.argsort(r).astype(np.int32)
    B = np.sort(order[:96])
    A = np.sort(order[-640:])
    assert r[A].min() > 4 * r[B].max()
    f = F(m, x, v, precision="mixed")
    out = f.accel_gradient(A, B, eps_grad=0.05)
    a_ref, g_ref = oracle_g(m, x, A, B)
    ea, eg = rel(cpu(out["acc"]), a_ref), rel(cpu(out["grad"]), g_ref)
    assert p999(ea) < 1e-6 and p999(eg) < 1e-6, (p999(ea), p999(eg))
    # the reverse pass, the core against the outskirts, also fills every slot; but the shell
    # of sources nearly cancels its own pull (sum_j |term| / |a| reaches 140 here), so it is
    # held to the bound of a floating-point sum: 1e-7 of the sum of the terms' magnitudes
    out = f.accel_gradient(B, A, eps_grad=0.05)
    a_ref, g_ref = oracle_g(m, x, B, A)
    a_src = oracle.acc(m, x, A, B)
    d = x[A][None, :, :] - x[B][:, None, :]
    ri = 1.0 / np.linalg.norm(d, axis=2)
    Sa = (m[A][None, :] * ri ** 2).sum(1)
    da = a_src[None, :, :] - a_ref[:, None, :]
    tg = (m[A][None, :] * ri ** 3)[..., None] * (da - 3.0 * ((d * da).sum(2) * ri ** 2)[..., None] * d)
    Sg = 2.0 * np.linalg.norm(tg, axis=2).sum(1)
    assert np.all(np.linalg.norm(cpu(out["acc"]) - a_ref, axis=1) < 1e-7 * Sa)
    assert np.all(np.linalg.norm(cpu(out["grad"]) - g_ref, axis=1) < 1e-7 * Sg)
    f.close()


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_accel_gradient_mixed_across_seeds(seed):
    """The mixed bar on four equal-mass Plummer spheres of N = 8192 (a full-set pass and a
    cross pass with |A| = N/4), so that the 99.9th percentile does not rest on one lucky
    draw.  The relative error of g_i is conditioned by sum_j |term_ij| / |g_i|, which is large
    where the gradient nearly vanishes; the dominant terms in double-float keep that tail
    near 5e-7 here."""
    n = 8192
    m, x, v = ics.plummer(n, seed)
    f = F(m, x, v, precision="mixed")
    A = np.arange(n, dtype=np.int32)
    out = f.accel_gradient(None, None, eps_grad=0.05)
    a_ref, g_ref = oracle_g(m, x, A, A)
    ea, eg = rel(cpu(out["acc"]), a_ref), rel(cpu(out["grad"]), g_ref)
    assert p999(ea) < 1e-6 and p999(eg) < 1e-6, (p999(ea), p999(eg))
    perm = np.random.default_rng(3).permutation(n).astype(np.int32)
    S, Fl = np.sort(perm[: n // 4]), perm[n // 4:]
    out = f.accel_gradient(S, Fl, eps_grad=0.05)
    a_ref, g_ref = oracle_g(m, x, S, Fl)
    ea, eg = rel(cpu(out["acc"]), a_ref), rel(cpu(out["grad"]), g_ref)
    assert p999(ea) < 1e-6 and p999(eg) < 1e-6, (p999(ea), p999(eg))
    f.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("cross", [False, True])
def test_accel_gradient_hard_binaries(precision, cross):
    """Plummer N = 8192 with Kroupa masses and 5% hard binaries (a = 1e-5..1e-3, thermal e):
    members' accelerations exceed the median by up to ~1e7 and the terms of the two partners
    cancel in every other particle's gradient, which amplifies FP32 rounding by the ratio of
    distances; the mixed pass sums these hot sources in double-float and must still meet 1e-6
    at the 99.9th percentile.  cross: disjoint lists that split binaries between them."""
    n = 8192
    m, x, v = ics.plummer_kroupa_binaries(n, 17)
    f = F(m, x, v, precision=precision)
    eps = 1e-3
    if cross:
        perm = np.random.default_rng(5).permutation(n).astype(np.int32)
        A, B = np.sort(perm[:2500]), perm[2500:]
        out = f.accel_gradient(A, B, eps_grad=eps)
    else:
        A = B = np.arange(n, dtype=np.int32)
        out = f.accel_gradient(None, None, eps_grad=eps)
    a_ref, g_ref = oracle_g(m, x, A, B)
    ea, eg = rel(cpu(out["acc"]), a_ref), rel(cpu(out["grad"]), g_ref)
    if precision == "fp64":
        # g of a particle near a tight pair is a sum whose terms cancel to ~1e-5 of their size,
        # so two FP64 summations differ by ~1e-16 of the sum of |terms|, not of |g|: the bound
        # is 1e-12 of that sum (the classical error bound of a floating-point sum)
        assert ea.max() < 1e-12, ea.max()
        g = cpu(out["grad"])
        bad = np.nonzero(eg > 1e-12)[0]
        if bad.size:
            aB = oracle.acc(m, x, np.asarray(B, dtype=np.int32), np.asarray(A, dtype=np.int32))
            Bi = np.asarray(B)
            for k in bad:
                d = x[Bi] - x[A[k]]
                da = aB - a_ref[k]
                r2 = (d * d).sum(1)
                ok = r2 > 0
                ri = 1.0 / np.sqrt(r2[ok])
                term = (m[Bi][ok] * ri ** 3)[:, None] * (
                    da[ok] - 3.0 * ((d[ok] * da[ok]).sum(1) * ri * ri)[:, None] * d[ok])
                S = 2.0 * np.linalg.norm(term, axis=1).sum()
                assert np.linalg.norm(g[k] - g_ref[k]) < 1e-12 * S, (k, eg[k])
    else:
        assert p999(ea) < 1e-6 and p999(eg) < 1e-6, (p999(ea), p999(eg))
        assert ea.max() < 1e-5 and eg.max() < 1e-5, (ea.max(), eg.max())
    f.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotune_keeps_results(precision):
    """The launch-shape autotuner only changes how the sources are split and which kernel
    layout runs: after it, a full acc + gradient pass still meets the parity bounds, and every
    size 512..N got a choice (negative: the small-tile layout, mixed mode only)."""
    n = 4096
    m, x, v = ics.plummer(n, 31, masses=ics.kroupa_masses(n, 31))
    f = F(m, x, v, precision=precision)
    table = f.autotune()
    # the Newtonian pass that feeds a gradient has a row of its own in the mixed mode
    kinds = ("acc", "grad", "tstep") + (("acc_feeding_grad",) if precision == "mixed" else ())
    assert precision == "mixed" or table["acc_feeding_grad"] == {}, table
    for kind in kinds:
        assert sorted(table[kind]) == [512, 1024, 2048, 4096], table
        assert all(abs(w) in (1, 2, 4, 8, 16) for w in table[kind].values())
        assert precision == "mixed" or all(w > 0 for w in table[kind].values())
    out = f.accel_gradient(None, None, eps_grad=0.01)
    A = np.arange(n, dtype=np.int32)
    a_ref, g_ref = oracle_g(m, x, A, A)
    ea, eg = rel(cpu(out["acc"]), a_ref), rel(cpu(out["grad"]), g_ref)
    if precision == "fp64":
        assert ea.max() < 1e-12 and eg.max() < 1e-12
    else:
        assert p999(ea) < 1e-6 and p999(eg) < 1e-6
    tau = cpu(f.timesteps())
    et = rel(tau, oracle.timesteps(m, x, v, A, eta=0.2))
    assert (et.max() < 1e-12) if precision == "fp64" else (p999(et) < 2e-6)
    f.close()


def test_accel_gradient_two_body_closed_form():
    """Pin on the GPU path itself: two bodies give a~ = (1 + eps^2 G M / (12 r^3)) a."""
    G = 1.3
    m, x, v = ics.kepler_binary(0.4, 1.1, 0.7, 0.2, G=G, mean_anomaly=0.8)
    for prec, tol in (("fp64", 1e-14), ("mixed", 1e-6)):
        f = F(m, x, v, G=G, precision=prec)
        out = f.accel_gradient(None, None, eps_grad=0.1)
        r = np.linalg.norm(x[0] - x[1])
        fac = 1 + 0.01 * G * m.sum() / (12 * r ** 3)
        a = cpu(out["acc"])
        assert rel(cpu(out["acc_tilde"]), fac * a).max() < tol
        assert rel(a[:1], (G * m[1] * (x[1] - x[0]) / r ** 3)[None]).max() < tol
        f.close()


def test_accel_gradient_edge_cases():
    from paper_2011_14984_gb300 import frost as fr
    m, x, v = ics.plummer(300, 5)
    f = F(m, x, v, precision="mixed")
    # empty active list
    out = f.accel_gradient(np.zeros(0, np.int32), np.arange(10, dtype=np.int32))
    assert out["acc"].shape == (0, 3)
    # empty source list: zero acceleration, a~ = a
    out = f.accel_gradient(np.arange(5, dtype=np.int32), np.zeros(0, np.int32), eps_grad=0.1)
    assert float(out["acc"].abs().max()) == 0.0 and float(out["grad"].abs().max()) == 0.0
    # single particle against itself
    out = f.accel_gradient(np.array([7], np.int32), np.array([7], np.int32), eps_grad=0.1)
    assert float(out["acc"].abs().max()) == 0.0
    # partial overlap, repeated and out-of-range indices are rejected
    with pytest.raises(fr.FrostError) as e:
        f.accel_gradient(np.array([1, 2, 3], np.int32), np.array([3, 4], np.int32))
    assert e.value.code == fr.FROST_EINVAL
    with pytest.raises(fr.FrostError) as e:
        f.accel_gradient(np.array([1, 1], np.int32), np.array([3, 4], np.int32))
    assert e.value.code == fr.FROST_EINVAL
    with pytest.raises(fr.FrostError) as e:
        f.accel_gradient(np.array([1, 2], np.int32), np.array([3, 400], np.int32))
    assert e.value.code == fr.FROST_EINVAL
    f.close()


def test_coincident_and_nonfinite_inputs_are_reported():
    from paper_2011_14984_gb300 import frost as fr
    m, x, v = ics.plummer(200, 6)
    x[17] = x[42]
    for prec in ("fp64", "mixed"):
        f = F(m, x, v, precision=prec)
        with pytest.raises(fr.FrostError) as e:
            f.accel_gradient(None, None, eps_grad=0.1)
        assert e.value.code == fr.FROST_ECOINCIDENT
        f.close()
        f = F(m, x, v, precision=prec)
        with pytest.raises(fr.FrostError) as e:
            f.timesteps()
        assert e.value.code == fr.FROST_ECOINCIDENT
        f.close()
    x[17, 0] = np.nan
    with pytest.raises(fr.FrostError) as e:
        F(m, x, v)
    assert e.value.code == fr.FROST_ENONFINITE


# ---------------------------------------------------------------------------------------
# time-steps, partition, kick / drift
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("sym", [0, 1, 2, 4, 5])
def test_timesteps(precision, sym):
    """Time-steps of a set with 10% binaries for each symmetrisation factor, with the
    two-body fly-by derivative (sym < 4) and the exact one (sym | 4: accelerations of the set
    due to itself, softened by eps_P)."""
    n = 2500
    m, x, v = ics.plummer_kroupa_binaries(n, 9, binary_fraction=0.1)
    eps = 1e-4 if sym & 4 else 0.0
    f = F(m, x, v, precision=precision, sym=sym, eta=0.2, eps_soft=eps)
    rng = np.random.default_rng(1)
    P = rng.permutation(n)[:1900].astype(np.int32)
    tau = cpu(f.timesteps(P))
    ref = oracle.timesteps_ex(m, x, v, P, P, eta=0.2, eps2=eps * eps, sym=sym)
    e = rel(tau, ref)
    if precision == "fp64":
        assert e.max() < 1e-12, e.max()
    else:
        assert p999(e) < 2e-6 and e.max() < 1e-4, (p999(e), e.max())
    assert np.isinf(cpu(f.timesteps(np.array([3], np.int32))))[0]
    f.close()


@pytest.mark.parametrize("sym", [0, 1, 2, 4, 5])
@pytest.mark.parametrize("n", [5000, 16384, 700])
def test_symmetric_timestep_pass_is_bit_identical(sym, n):
    """The symmetric time-step pass (each pair once for both particles: the pair criteria are
    symmetric bit for bit and the minimum does not depend on the order; the skip bound is the
    larger of the two particles' bounds) gives the one-sided pass's tau bit for bit, for every
    symmetrisation and the exact fly-by derivative, on ragged sizes; and both match the
    oracle within the mixed tolerance."""
    m, x, v = ics.plummer(n, 30 + n % 11, masses=ics.kroupa_masses(n, 30 + n % 11))
    out = {}
    for sc in (1, -1):
        f = F(m, x, v, precision="mixed", eta=0.2, sym=sym, sym_cross=sc)
        out[sc] = cpu(f.timesteps())
        f.close()
    assert np.array_equal(out[1], out[-1]), np.max(np.abs(out[1] - out[-1]) / out[-1])
    I = np.sort(np.random.default_rng(n).choice(n, min(n, 256), replace=False)).astype(np.int32)
    ref = oracle.timesteps_ex(m, x, v, I, np.arange(n, dtype=np.int32), eta=0.2, sym=sym)
    assert p999(rel(out[1][I], ref)) < 2e-6


def test_timesteps_circular_binary_rule_of_thumb():
    """Eq. eta-two-pi on the GPU: tau = eta P / (2 pi) for a circular binary."""
    m, x, v = ics.kepler_binary(0.5, 0.5, 1.0, 0.0)
    for prec, tol in (("fp64", 1e-14), ("mixed", 2e-6)):
        f = F(m, x, v, precision=prec, eta=0.1)
        tau = cpu(f.timesteps())
        assert rel(tau, np.full(2, 0.1 * 2 * math.pi / (2 * math.pi))).max() < tol
        f.close()


def test_partition_bit_exact():
    m, x, v = ics.plummer(3000, 2)
    f = F(m, x, v)
    rng = np.random.default_rng(4)
    P = rng.permutation(3000)[:2777].astype(np.int32)
    tau = rng.random(2777)
    tau[::7] = 0.5  # ties go to the slow set
    for piv in (0.5, 0.0, 2.0, 0.123):
        S, Fl = f.partition(P, tau, piv)
        Sr, Fr = oracle.partition(P, tau, piv)
        assert np.array_equal(cpu(S), Sr) and np.array_equal(cpu(Fl), Fr)
    S, Fl = f.partition(P[:0], tau[:0], 0.5)
    assert S.numel() == 0 and Fl.numel() == 0
    f.close()


@pytest.mark.parametrize("n", [8192, 12289, 65536])
def test_partition_of_large_sets_bit_exact(n):
    """Sets of 8192 and more are split by many blocks (per-block slow counts, then a scatter
    from each block's offsets): the same lists as the oracle's stable partition, ties to the
    slow set, at a multiple of the block's 4096 entries and with a ragged last block."""
    m, x, v = ics.plummer(n + 100, 3)
    f = F(m, x, v)
    rng = np.random.default_rng(n)
    P = rng.permutation(n + 100)[:n].astype(np.int32)
    tau = rng.random(n)
    tau[::7] = 0.5
    for piv in (0.5, 0.0, 2.0, 0.123):
        S, Fl = f.partition(P, tau, piv)
        Sr, Fr = oracle.partition(P, tau, piv)
        assert np.array_equal(cpu(S), Sr) and np.array_equal(cpu(Fl), Fr), piv
    f.close()


def test_kick_drift_bit_exact():
    n = 1000
    m, x, v = ics.plummer(n, 8)
    f = F(m, x, v, precision="fp64")
    rng = np.random.default_rng(2)
    I = rng.permutation(n)[:600].astype(np.int32)
    a = rng.standard_normal((600, 3))
    f.kick(I, a, 0.0123)
    f.drift(I, 0.031)
    xg, vg, _ = f.state()
    xo, vo = x.copy(), v.copy()
    oracle.kick(I, vo, a, 0.0123)
    oracle.drift(I, xo, vo, 0.031)
    assert np.array_equal(xg, xo) and np.array_equal(vg, vo)
    f.close()


# ---------------------------------------------------------------------------------------
# integrator
# ---------------------------------------------------------------------------------------

def test_fsi_step_parity():
    n = 700
    m, x, v = ics.plummer(n, 12)
    S = np.arange(0, n, 2, dtype=np.int32)
    f = F(m, x, v, precision="fp64")
    f.fsi(S, 1e-2)
    xg, vg, _ = f.state()
    xo, vo = oracle.fsi(m, x, v, S, 1e-2)
    assert np.max(np.abs(xg - xo)) < 1e-14 and np.max(np.abs(vg - vo)) < 1e-12


@pytest.mark.parametrize("sym", [0, 4])
def test_hhs_fsi_trajectory_parity_fp64(sym):
    """Plummer N = 1024 (seed 1) to t = 0.125 in 16 top-level steps of 2^-7, eta = 0.2:
    positions within 1e-10 of the oracle and the same hierarchy depth (sym 4: the exact
    fly-by derivative)."""
    m, x, v = ics.plummer(1024, 1)
    f = F(m, x, v, precision="fp64", eta=0.2, sym=sym)
    f.step(2.0 ** -7, 16)
    xg, vg, t = f.state()
    st = f.stats()
    oracle.reset_counters()
    xo, vo = oracle.steps(m, x, v, 2.0 ** -7, 16, eta=0.2, sym=sym)
    oc = oracle.counters()
    assert t == pytest.approx(0.125)
    assert np.max(np.abs(xg - xo)) < 1e-10 and np.max(np.abs(vg - vo)) < 1e-9
    assert st["max_depth_seen"] == oc["max_depth"]
    e_g, e_o = f.energy(), oracle.energy(m, xo, vo)
    assert abs(e_g["E"] - e_o["E"]) < 1e-12 * abs(e_o["E"])
    f.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_symmetric_kick_sf_trajectory(precision):
    """The kick_sf of every level with each S x F pair once (sym_cross = 1, at every size; the
    force-gradient kick too in mixed mode): Plummer N = 1024 to t = 0.125 as in the serial test
    above, FP64 within 1e-10 of the
    oracle and the same depth; mixed within the mixed tolerance of the grid-path comparison
    (1e-7 in position) of the run with two one-sided passes, and the same depth."""
    m, x, v = ics.plummer(1024, 1)
    f = F(m, x, v, precision=precision, eta=0.2, sym_cross=1)
    f.step(2.0 ** -7, 16)
    xg, vg, _ = f.state()
    st = f.stats()
    f.close()
    assert st["acc_pairs_symmetric"] > 0
    assert (st["grad_pairs_symmetric"] > 0) == (precision == "mixed")
    if precision == "fp64":
        oracle.reset_counters()
        xo, vo = oracle.steps(m, x, v, 2.0 ** -7, 16, eta=0.2)
        assert np.max(np.abs(xg - xo)) < 1e-10 and np.max(np.abs(vg - vo)) < 1e-9
        assert st["max_depth_seen"] == oracle.counters()["max_depth"]
    else:
        g = F(m, x, v, precision=precision, eta=0.2, sym_cross=-1)
        g.step(2.0 ** -7, 16)
        x2, _, _ = g.state()
        st2 = g.stats()
        g.close()
        assert st2["acc_pairs_symmetric"] == 0 and st2["max_depth_seen"] == st["max_depth_seen"]
        assert np.max(np.abs(xg - x2)) < 1e-7, np.max(np.abs(xg - x2))


def test_hold2_integrator_trajectory_parity_fp64():
    """The second-order HOLD integrator (Eq. hhs2) on the GPU kernels: Plummer N = 1024,
    8 top-level steps of 2^-7, FP64 positions within 1e-10 of the oracle's HOLD, the same
    depth; and it differs from the fourth-order HHS-FSI run (a different integrator)."""
    from paper_2011_14984_gb300.frost import FROST_HOLD2
    m, x, v = ics.plummer(1024, 1)
    f = F(m, x, v, precision="fp64", eta=0.2, integrator=FROST_HOLD2)
    f.step(2.0 ** -7, 8)
    xg, vg, t = f.state()
    st = f.stats()
    oracle.reset_counters()
    xo, vo = oracle.steps_hold(m, x, v, 2.0 ** -7, 8, eta=0.2)
    oc = oracle.counters()
    assert np.max(np.abs(xg - xo)) < 1e-10 and np.max(np.abs(vg - vo)) < 1e-9
    assert st["max_depth_seen"] == oc["max_depth"]
    x4, _ = oracle.steps(m, x, v, 2.0 ** -7, 8, eta=0.2)
    assert np.max(np.abs(x4 - xo)) > 1e-9
    f.close()


def test_hhs_fsi_mixed_energy_parity():
    """Mixed precision reaches the FP64 energy error within a factor 2 (plus round-off)."""
    m, x, v = ics.plummer(1024, 1)
    E0 = oracle.energy(m, x, v)["E"]
    dE = {}
    for prec in ("fp64", "mixed"):
        f = F(m, x, v, precision=prec, eta=0.2)
        f.step(2.0 ** -7, 16)
        dE[prec] = abs((f.energy()["E"] - E0) / E0)
        f.close()
    assert dE["mixed"] < 2 * dE["fp64"] + 1e-11, dE


@pytest.mark.parametrize("precision,n,subtree_max", [("mixed", 16384, 0), ("mixed", 4096, 64),
                                                      ("fp64", 4096, 100)])
def test_concurrent_branches_are_bit_identical_to_the_serial_order(precision, n, subtree_max):
    """fsi(S) of every grid-level hhs_fsi call runs on a stream of its own, concurrently with
    hhs_fsi(F) (disjoint particles): the state after two steps is the serial order's bit for
    bit, with the same pair counts and depth; small subtree thresholds put several grid
    levels (several branch streams) in flight at once."""
    m, x, v = ics.plummer(n, 40 + n % 7)
    out = {}
    for branch in (0, -1):
        f = F(m, x, v, precision=precision, eta=0.2, subtree_max=subtree_max, branch_streams=branch)
        f.step(2.0 ** -7, 2)
        xg, vg, _ = f.state()
        st = f.stats()
        out[branch] = (xg, vg, st["acc_pairs"], st["grad_pairs"], st["max_depth_seen"], st["hhs_calls"])
        f.close()
    assert out[0][4] >= 3
    assert np.array_equal(out[0][0], out[-1][0]) and np.array_equal(out[0][1], out[-1][1])
    assert out[0][2:] == out[-1][2:]


def test_solar_system_hhs_fsi_on_gpu():
    """The paper's five-body initial state (App. A1) through frost_step in FP64: the same
    trajectory as the oracle after 200 years at eta = 0.05."""
    from conftest import load_solar_system
    _, m, x, v, G = load_solar_system()
    f = F(m, x, v, G=G, eta=0.05, precision="fp64")
    n = int(round(200 * 365.25 / 4096.0))
    f.step(4096.0, n)
    xg, vg, _ = f.state()
    xo, vo = oracle.steps(m, x, v, 4096.0, n, G=G, eta=0.05)
    assert np.max(np.abs(xg - xo)) < 1e-9
    f.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("e", [0.0, 0.9])
def test_equal_mass_binary_conserves_momentum_exactly(precision, e):
    """The paper's binary experiment (Sec. 6.1.1): with two equal masses the two kicks of
    every step are exact negatives (x_j - x_i = -(x_i - x_j), the same r^2 and weights), so the
    total momentum stays exactly zero over many orbits, in both precision modes."""
    m, x, v = ics.kepler_binary(1.0, 1.0, 1.0, e)
    P0 = (m[:, None] * v).sum(0)
    assert np.all(P0 == 0.0)
    f = F(m, x, v, precision=precision, eta=0.05)
    f.step(2.0 ** -5, 200)
    xg, vg, _ = f.state()
    assert np.all((m[:, None] * vg).sum(0) == 0.0), (m[:, None] * vg).sum(0)
    f.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checkpoint_restart_is_bit_identical(precision, tmp_path):
    """Checkpoint / restart through the snapshot-as-initial-condition route: 4 + 4 steps with
    the state written to disk and read into a fresh context give the same bits as 8 steps
    in one context (the step depends only on the state: no history is carried)."""
    m, x, v = ics.plummer(3000, 61, masses=ics.kroupa_masses(3000, 61))
    dt = 2.0 ** -7
    f = F(m, x, v, precision=precision)
    f.step(dt, 8)
    x8, v8, t8 = f.state()
    f.close()
    g = F(m, x, v, precision=precision)
    g.step(dt, 4)
    xs, vs, ts = g.state()
    g.close()
    path = tmp_path / "snapshot.npz"
    np.savez(path, m=m, x=xs, v=vs, t=ts)
    snap = np.load(path)
    h = F(snap["m"], snap["x"], snap["v"], precision=precision)
    h.set_state(snap["x"], snap["v"], float(snap["t"]))
    h.step(dt, 4)
    xr, vr, tr = h.state()
    h.close()
    assert tr == t8
    assert np.array_equal(xr, x8) and np.array_equal(vr, v8)


def test_energy_momentum_parity():
    """E, P, L against the oracle; the potential runs in double-float arithmetic on the GPU,
    so U is also checked where hard binaries (separations down to 1e-5) dominate it."""
    n = 3000
    m, x, v = ics.plummer(n, 77, masses=ics.kroupa_masses(n, 77))
    mb, xb, vb = ics.plummer_kroupa_binaries(8192, 17)
    for (mm, xx, vv), eps in (((m, x, v), 0.0), ((m, x, v), 0.01), ((mb, xb, vb), 0.0)):
        f = F(mm, xx, vv, eps_soft=eps)
        e = f.energy()
        r = oracle.energy(mm, xx, vv, eps2=eps * eps)
        assert abs(e["T"] - r["T"]) < 1e-13 * abs(r["T"])
        assert abs(e["U"] - r["U"]) < 1e-12 * abs(r["U"]), (e["U"], r["U"])
        assert np.max(np.abs(e["P"] - r["P"])) < 1e-15
        assert np.max(np.abs(e["L"] - r["L"])) < 1e-14
        f.close()


def test_depth_limit():
    from paper_2011_14984_gb300 import frost as fr
    m, x, v = ics.kepler_binary(0.5, 0.5, 1e-3, 0.0)
    f = F(m, x, v, max_depth=3)
    with pytest.raises(fr.FrostError) as e:
        f.step(1.0, 1)
    assert e.value.code == fr.FROST_EDEPTH
    f.close()


# ---------------------------------------------------------------------------------------
# full-size launch configurations, checked on sampled particles
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_full_pass_64k_sampled(precision):
    """Plummer N = 65536 (seed 2), the full acc + gradient pass of the benchmark: 512
    sampled particles against the oracle, which computes every a_j for the gradient."""
    m, x, v = ics.workload("plummer_64k")
    n = m.size
    f = F(m, x, v, precision=precision)
    eps = 2.0 ** -8
    out = f.accel_gradient(None, None, eps_grad=eps)
    rng = np.random.default_rng(11)
    I = np.sort(rng.choice(n, 512, replace=False)).astype(np.int32)
    A = np.arange(n, dtype=np.int32)
    a_all = oracle.acc(m, x, A, A)
    g_ref = oracle.grad(m, x, I, a_all[I], A, a_all)
    ea = rel(cpu(out["acc"])[I], a_all[I])
    eg = rel(cpu(out["grad"])[I], g_ref)
    if precision == "fp64":
        assert ea.max() < 1e-12 and eg.max() < 1e-12
    else:
        assert p999(ea) < 1e-6 and p999(eg) < 1e-6, (p999(ea), p999(eg))
    # a property at any size: total force vanishes
    a = cpu(out["acc"])
    Ftot = (m[:, None] * a).sum(0)
    assert np.all(np.abs(Ftot) < 1e-9 * (m[:, None] * np.abs(a)).sum())
    f.close()


# ---------------------------------------------------------------------------------------
# single-block subtree solver (hhs_fsi subtrees of small sets in one thread block)
# ---------------------------------------------------------------------------------------

def test_full_pass_64k_every_particle_mixed():
    """The mixed bar at the benchmark's size over every particle, not a sample: Plummer
    N = 65536 (the benchmark sphere), the full-set acc + gradient pass against the oracle's
    a and g of all 65536 particles."""
    m, x, v = ics.workload("plummer_64k")
    n = m.size
    f = F(m, x, v, precision="mixed")
    out = f.accel_gradient(None, None, eps_grad=2.0 ** -7)
    A = np.arange(n, dtype=np.int32)
    a_ref, g_ref = oracle_g(m, x, A, A)
    ea, eg = rel(cpu(out["acc"]), a_ref), rel(cpu(out["grad"]), g_ref)
    assert p999(ea) < 1e-6 and p999(eg) < 1e-6, (p999(ea), p999(eg))
    f.close()


@pytest.mark.parametrize("subtree_max", [1 << 30, 100])
@pytest.mark.parametrize("sym", [0, 4])
def test_subtree_solver_trajectory_parity_fp64(subtree_max, sym):
    """Whole recursion in one block (1<<30) or only sets of <= 100 particles: the same
    trajectory as the oracle (Plummer N = 700, 6 top-level steps of 2^-7, eta = 0.2), with
    the two-body (sym 0) or the exact (sym 4) fly-by derivative."""
    m, x, v = ics.plummer(700, 31, masses=ics.kroupa_masses(700, 31))
    f = F(m, x, v, precision="fp64", eta=0.2, subtree_max=subtree_max, sym=sym)
    f.step(2.0 ** -7, 6)
    xg, vg, _ = f.state()
    st = f.stats()
    oracle.reset_counters()
    xo, vo = oracle.steps(m, x, v, 2.0 ** -7, 6, eta=0.2, sym=sym)
    oc = oracle.counters()
    assert st["subtree_launches"] > 0
    assert np.max(np.abs(xg - xo)) < 1e-10 and np.max(np.abs(vg - vo)) < 1e-9
    assert st["max_depth_seen"] == oc["max_depth"]
    f.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_subtree_solver_fsi_beside_the_warp_path_is_bit_identical(precision):
    """Inside the single-block solver, a set's two fsi(S, tau/2) steps run on warps 1..7 while
    warp 0 advances the fast set F (at most 32 particles) through hhs_fsi(F, tau/2): H_S and H_F
    act on disjoint particles (Algorithm hhs-fsi).  The whole recursion of a 700-particle
    Kroupa sphere in one block, 6 top-level steps: the state is the serial order's
    (branch_streams = -1) bit for bit, with the same pair counts and depth; the overlap ran;
    and FP64 stays within the oracle's 1e-10."""
    m, x, v = ics.plummer(700, 31, masses=ics.kroupa_masses(700, 31))
    out = {}
    for branch in (0, -1):
        f = F(m, x, v, precision=precision, eta=0.2, subtree_max=1 << 30, branch_streams=branch)
        f.step(2.0 ** -7, 6)
        xg, vg, _ = f.state()
        st = f.stats()
        out[branch] = (xg, vg, st)
        f.close()
    st0, st1 = out[0][2], out[-1][2]
    assert st0["subtree_launches"] == 6 and st0["subtree_fsi_beside"] > 0, st0["subtree_fsi_beside"]
    assert st1["subtree_fsi_beside"] == 0
    assert np.array_equal(out[0][0], out[-1][0]) and np.array_equal(out[0][1], out[-1][1])
    for k in ("acc_pairs", "grad_pairs", "tstep_pairs", "hhs_calls", "fsi_calls", "acc_pairs_reused",
              "max_depth_seen"):
        assert st0[k] == st1[k], k
    if precision == "fp64":
        xo, vo = oracle.steps(m, x, v, 2.0 ** -7, 6, eta=0.2)
        assert np.max(np.abs(out[0][0] - xo)) < 1e-10 and np.max(np.abs(out[0][1] - vo)) < 1e-9


def test_cluster_batch_fsi_beside_the_warp_path_is_bit_identical():
    """The batch teams of one block take the same overlap: a mixed-precision batch of six
    clusters of 40 to 300 particles, after one captured and one replayed step, equals the
    serial order bit for bit."""
    off, m, x, v = _small_batch()
    out = {}
    for branch in (0, -1):
        f = F(m, x, v, precision="mixed", eta=0.2, offsets=off, branch_streams=branch)
        f.step(2.0 ** -6, 1)
        f.step(2.0 ** -6, 1)
        out[branch] = f.state()[:2] + (f.stats()["subtree_fsi_beside"],)
        f.close()
    assert out[0][2] > 0 and out[-1][2] == 0
    assert np.array_equal(out[0][0], out[-1][0]) and np.array_equal(out[0][1], out[-1][1])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_subtree_solver_on_a_block_cluster(precision):
    """A single-set solver launch spread over an 8-block thread-block cluster (cluster
    barriers, the group path for every pass): the trajectory of the one-block solver, to the
    oracle's 1e-10 in FP64 and to the mixed-precision level otherwise."""
    m, x, v = ics.plummer(700, 31, masses=ics.kroupa_masses(700, 31))
    out = {}
    for blocks in (1, 8):
        f = F(m, x, v, precision=precision, eta=0.2, subtree_max=1 << 30, subtree_blocks=blocks)
        f.step(2.0 ** -7, 6)
        out[blocks] = f.state()[0]
        assert f.stats()["subtree_launches"] == 6
        f.close()
    if precision == "fp64":
        xo, _ = oracle.steps(m, x, v, 2.0 ** -7, 6, eta=0.2)
        assert np.max(np.abs(out[8] - xo)) < 1e-10
    else:
        assert np.max(np.abs(out[8] - out[1])) < 1e-7


def test_subtree_solver_mixed_matches_grid_path():
    """Mixed precision: the same steps with and without the single-block solver agree to
    the mixed-precision level and reach the same energy error."""
    m, x, v = ics.plummer(1024, 1)
    E0 = oracle.energy(m, x, v)["E"]
    out = {}
    for sm in (-1, 1 << 30):
        f = F(m, x, v, precision="mixed", eta=0.2, subtree_max=sm)
        f.step(2.0 ** -7, 4)
        xg, vg, _ = f.state()
        out[sm] = (xg, abs((f.energy()["E"] - E0) / E0), f.stats())
        f.close()
    assert out[1 << 30][2]["subtree_launches"] == 4 and out[-1][2]["subtree_launches"] == 0
    assert np.max(np.abs(out[-1][0] - out[1 << 30][0])) < 1e-7
    dEa, dEb = out[-1][1], out[1 << 30][1]
    assert max(dEa, dEb) < 2 * min(dEa, dEb) + 1e-12


def test_subtree_solver_depth_limit():
    from paper_2011_14984_gb300 import frost as fr
    m, x, v = ics.kepler_binary(0.5, 0.5, 1e-3, 0.0)
    f = F(m, x, v, max_depth=3, subtree_max=1 << 30)
    with pytest.raises(fr.FrostError) as e:
        f.step(1.0, 1)
    assert e.value.code == fr.FROST_EDEPTH
    f.close()


# ---------------------------------------------------------------------------------------
# batch of independent clusters (one thread block per cluster)
# ---------------------------------------------------------------------------------------

def _small_batch():
    sizes = [40, 97, 128, 64, 211, 300]
    ms, xs, vs = [], [], []
    for k, n in enumerate(sizes):
        m, x, v = ics.plummer(n, 500 + k)
        ms.append(m); xs.append(x); vs.append(v)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    return off, np.concatenate(ms), np.concatenate(xs), np.concatenate(vs)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cluster_batch_with_block_teams(precision):
    """A batch with clusters of at least 768 particles: those run on a thread-block cluster of
    8 blocks (cluster barriers between the passes), concurrently with the one-block clusters;
    every cluster still evolves as if alone."""
    sizes = [1500, 60, 900, 200, 800]
    ms, xs, vs = [], [], []
    for k, n in enumerate(sizes):
        m, x, v = ics.plummer(n, 700 + k)
        ms.append(m); xs.append(x); vs.append(v)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    m, x, v = np.concatenate(ms), np.concatenate(xs), np.concatenate(vs)
    f = F(m, x, v, precision=precision, eta=0.2, offsets=off)
    f.step(2.0 ** -6, 1)  # captures the batch step as a CUDA graph
    f.step(2.0 ** -6, 1)  # replays it
    xg, vg, t = f.state()
    st = f.stats()
    assert st["max_depth_seen"] >= 1
    tol = 1e-10 if precision == "fp64" else 1e-7
    for k in range(len(sizes)):
        a, b = off[k], off[k + 1]
        xo, vo = oracle.steps(m[a:b], x[a:b], v[a:b], 2.0 ** -6, 2, eta=0.2)
        assert np.max(np.abs(xg[a:b] - xo)) < tol, (k, np.max(np.abs(xg[a:b] - xo)))
    f.close()


def test_cluster_batch_autotuned_team_split_keeps_results():
    """frost_autotune on a batch context picks the team split (which clusters run on a
    thread-block cluster of several blocks) by timing one step of every candidate from the same
    state; it restores the state and time, and the tuned context still evolves every cluster as
    the oracle does (FP64, 1e-10)."""
    sizes = [1500, 60, 900, 200, 800, 3000]
    ms, xs, vs = [], [], []
    for k, n in enumerate(sizes):
        m, x, v = ics.plummer(n, 720 + k)
        ms.append(m); xs.append(x); vs.append(v)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    m, x, v = np.concatenate(ms), np.concatenate(xs), np.concatenate(vs)
    f = F(m, x, v, precision="fp64", eta=0.2, offsets=off)
    tuned = f.autotune()
    assert tuned["team_blocks"] in (1, 2, 4, 8) and tuned["team_min_n"] >= 256
    x0, v0, t0 = f.state()
    assert t0 == 0.0 and np.array_equal(x0, x) and np.array_equal(v0, v)
    f.step(2.0 ** -6, 1)
    xg, _, _ = f.state()
    f.close()
    for k in range(len(sizes)):
        a, b = off[k], off[k + 1]
        xo, _ = oracle.steps(m[a:b], x[a:b], v[a:b], 2.0 ** -6, 1, eta=0.2)
        assert np.max(np.abs(xg[a:b] - xo)) < 1e-10, (k, np.max(np.abs(xg[a:b] - xo)))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cluster_batch_matches_oracle_per_cluster(precision):
    """frost_init_batch + frost_step: every cluster evolves as if alone (the oracle runs each
    cluster separately): FP64 positions within 1e-10, mixed within 1e-7, and the per-cluster
    energies agree with the oracle's."""
    off, m, x, v = _small_batch()
    f = F(m, x, v, precision=precision, eta=0.2, offsets=off)
    f.step(2.0 ** -6, 3)
    xg, vg, t = f.state()
    ecl = f.cluster_energies()
    st = f.stats()
    assert st["max_depth_seen"] >= 1
    tol = 1e-10 if precision == "fp64" else 1e-7
    for k in range(off.size - 1):
        a, b = off[k], off[k + 1]
        xo, vo = oracle.steps(m[a:b], x[a:b], v[a:b], 2.0 ** -6, 3, eta=0.2)
        assert np.max(np.abs(xg[a:b] - xo)) < tol, (k, np.max(np.abs(xg[a:b] - xo)))
        eo = oracle.energy(m[a:b], xg[a:b], vg[a:b])
        assert abs(ecl["E"][k] - eo["E"]) < 1e-12 * abs(eo["E"])
        assert np.max(np.abs(ecl["P"][k] - eo["P"])) < 1e-14
    tot = f.energy()
    assert abs(tot["E"] - ecl["E"].sum()) < 1e-12 * abs(ecl["E"].sum())
    f.close()


def test_full_cluster_batch_fp64_one_step_sampled_clusters():
    """The full 256-cluster batch (N log-uniform in 64..4096, 232818 particles) in FP64: one
    top-level step of 2^-7 of every cluster in one launch; 16 sampled clusters (the largest
    and the smallest among them) evolve as the oracle evolves each of them alone, positions
    within 1e-10 and velocities within 1e-9, and every cluster keeps its momentum."""
    off, m, x, v = ics.batch_workload("cluster_batch_256")
    sz = np.diff(off)
    f = F(m, x, v, precision="fp64", eta=0.2, offsets=off)
    p0 = f.cluster_energies()["P"]
    f.step(2.0 ** -7, 1)
    xg, vg, t = f.state()
    p1 = f.cluster_energies()["P"]
    f.close()
    assert t == pytest.approx(2.0 ** -7)
    rng = np.random.default_rng(5)
    pick = np.unique(np.concatenate([[int(np.argmax(sz)), int(np.argmin(sz))],
                                     rng.choice(sz.size, 14, replace=False)]))
    assert pick.size >= 15
    for k in pick:
        a, b = off[k], off[k + 1]
        xo, vo = oracle.steps(m[a:b], x[a:b], v[a:b], 2.0 ** -7, 1, eta=0.2)
        assert np.max(np.abs(xg[a:b] - xo)) < 1e-10, (k, sz[k], np.max(np.abs(xg[a:b] - xo)))
        assert np.max(np.abs(vg[a:b] - vo)) < 1e-9, (k, sz[k], np.max(np.abs(vg[a:b] - vo)))
    assert np.max(np.abs(p1 - p0)) < 1e-14


def test_mixed_gradient_beyond_the_fp32_range_at_a_binary_pericentre():
    """A Kroupa sphere (N = 2000) with two members 7e-11 apart, the pericentre of the tightest
    binary of the 262k hard-binary workload (a = 1.6e-5, e = 0.999996): their mutual gradient
    term, m r^-5 |r^2 a_ji - 3 (x.a) x| ~ 1e45, is beyond the largest FP32 value (3.4e38), so
    the double-float evaluation of that dominant term overflows and the library evaluates it in
    FP64.  The pass stays finite; a meets the mixed bars for every particle, and the two
    members' g is within 1e-5 of the oracle (the 48-bit split records resolve their
    separation to ~3e-7 of itself, and g ~ r^-3).

    For every other particle the two members' gradient terms (~2e15 each at distance 0.1)
    cancel to ~1e4, a ratio of ~4e-12, so no arithmetic of fewer than ~80 bits resolves them:
    the FP64 oracle itself carries ~1e-4 there.  g is held to the classical bound of a sum
    whose terms are rounded to the 2^-40 of the double-float hot-source path (reading 17):
    |dg_i| <= 1e-6 |g_i| + 2^-40 sum_j |term_ij|."""
    m, x, v = ics.plummer(2000, 77, masses=ics.kroupa_masses(2000, 77))
    d = np.random.default_rng(1).normal(size=3)
    x[1] = x[0] + 7e-11 * d / np.linalg.norm(d)
    A = np.arange(m.size, dtype=np.int32)
    a_ref, g_ref = oracle_g(m, x, A, A)
    f = F(m, x, v, precision="mixed")
    out = f.accel_gradient(None, None, eps_grad=2.0 ** -20)
    f.close()
    a, g = cpu(out["acc"]), cpu(out["grad"])
    assert np.isfinite(a).all() and np.isfinite(g).all()
    assert np.linalg.norm(g_ref[:2], axis=1).min() > 1e40  # the case is out of the FP32 range
    ea, eg = rel(a, a_ref), rel(g, g_ref)
    assert p999(ea) < 1e-6 and ea.max() < 1e-5, (p999(ea), ea.max())
    assert eg[:2].max() < 1e-5, eg[:2]
    # sum over j of |term_ij| of every particle's gradient (2 G prefactor included)
    S = np.zeros(m.size)
    for k0 in range(0, m.size, 250):
        I = np.arange(k0, min(m.size, k0 + 250))
        dx = x[None, :, :] - x[I, None, :]
        da = a_ref[None, :, :] - a_ref[I, None, :]
        r2 = (dx * dx).sum(-1)
        r2[np.arange(I.size), I] = np.inf
        ri2 = 1.0 / r2
        t = (m[None, :] * ri2 * np.sqrt(ri2))[..., None] * (da - 3.0 * ((dx * da).sum(-1) * ri2)[..., None] * dx)
        S[I] = 2.0 * np.linalg.norm(t, axis=-1).sum(1)
    dg = np.linalg.norm(g - g_ref, axis=1)[2:]
    bound = (1e-6 * np.linalg.norm(g_ref, axis=1) + 2.0 ** -40 * S)[2:]
    assert np.all(dg <= bound), (np.max(dg / bound), int(np.argmax(dg / bound)) + 2)


def test_mixed_gradient_of_tight_pairs_far_from_the_origin():
    """Pairs 1e-9 to 3e-6 apart at |x| = 1 to 4 (hard binaries near pericentre away from the
    centre): their mutual gradient term is a dominant, deferred double-float term built from
    12 + 12 + 24-bit split records.  For such pairs the high and middle parts cancel and the
    low-part difference is as large as the result, so the separation must be renormalised
    before it enters double-float products (an unnormalised one gave errors of 1e3 in r^2).
    Every member's a and g within 1e-5 of the oracle."""
    m, x, v = ics.plummer(1000, 81, masses=ics.kroupa_masses(1000, 81))
    rng = np.random.default_rng(2)
    seps = [1e-9, 3e-9, 1e-8, 3e-8, 1e-7, 3e-7, 1e-6, 3e-6]
    members = []
    for k, r in enumerate(seps):
        i, j = 2 * k, 2 * k + 1
        d = rng.normal(size=3)
        u = rng.normal(size=3)
        x[i] = (1.0 + 3.0 * k / len(seps)) * u / np.linalg.norm(u)
        x[j] = x[i] + r * d / np.linalg.norm(d)
        members += [i, j]
    A = np.arange(m.size, dtype=np.int32)
    a_ref, g_ref = oracle_g(m, x, A, A)
    f = F(m, x, v, precision="mixed")
    out = f.accel_gradient(None, None, eps_grad=1e-9)
    f.close()
    a, g = cpu(out["acc"]), cpu(out["grad"])
    ea, eg = rel(a, a_ref)[members], rel(g, g_ref)[members]
    assert ea.max() < 1e-5 and eg.max() < 1e-5, (ea.max(), eg.max(), np.round(np.log10(eg + 1e-30), 1))


def test_kroupa_hard_binaries_trajectory_fp64():
    """Plummer N = 2000 with Kroupa masses and 5 % hard binaries (a in [1e-5, 1e-3], thermal
    e; seed 31): one top-level step of 2^-10 reaches hierarchy depth 19, through the grid
    levels, the single-block subtree solver and its one-warp path.

    Tolerance.  Over the ~2^19 sub-steps of the hardest binaries, FP64 round-off is amplified
    along the orbits: the oracle run on the same particles relabelled in reverse order (the
    same arithmetic, every sum in another order) differs from the oracle by ~6e-6 in the
    velocity of a binary member at ~6 (a relative error of 1e-6 in the binary's separation),
    while positions agree to 1e-11.  So: the same depth; positions within 1e-10; velocities
    within 4x the oracle's own spread under that relabelling (and within 1e-12 of it for the
    particles outside binaries, whose orbits are regular)."""
    m, x, v = ics.plummer_kroupa_binaries(2000, 31)
    n = m.size
    f = F(m, x, v, precision="fp64", eta=0.2)
    f.step(2.0 ** -10, 1)
    xg, vg, _ = f.state()
    st = f.stats()
    f.close()
    oracle.reset_counters()
    xo, vo = oracle.steps(m, x, v, 2.0 ** -10, 1, eta=0.2)
    oc = oracle.counters()
    rev = np.arange(n)[::-1]
    xr, vr = oracle.steps(m[rev], x[rev], v[rev], 2.0 ** -10, 1, eta=0.2)
    xr, vr = xr[rev], vr[rev]
    spread_v = np.max(np.abs(vr - vo))
    assert st["max_depth_seen"] == oc["max_depth"] >= 15, (st["max_depth_seen"], oc["max_depth"])
    assert np.max(np.abs(xg - xo)) < 1e-10, np.max(np.abs(xg - xo))
    assert np.max(np.abs(vg - vo)) <= 4.0 * spread_v, (np.max(np.abs(vg - vo)), spread_v)
    n_single = n - 2 * int(round(0.05 * n / 2.0))
    assert np.max(np.abs(vg[:n_single] - vo[:n_single])) < 1e-12


def test_kroupa_hard_binaries_mixed_integration_matches_fp64():
    """Mixed precision through the whole hierarchy of a sphere with hard binaries: Plummer
    N = 4096 with Kroupa masses and 5 % hard binaries (seed 31), one top-level step of 2^-10.
    It runs the grid levels with their hot-source gradient path (the binary members' large
    accelerations), the subtree solver and its one-warp path down to depth ~23.  It is compared
    with the same step in FP64 on the GPU.

    Tolerances.  The two runs reach the same depth, and the mixed energy error is within 2x of
    the FP64 one (the criterion for mixed precision).  The single stars move regularly.  An
    acceleration error eps |a| held over the step moves v by eps |a| t and x by eps |a| t^2 / 2.
    With eps = 2e-7 (the mixed pass's 99.9th percentile) and A = 2x the 99th percentile of the
    singles' |a| at t = 0, this bounds the 99.9th percentiles of their deviations.  With
    eps = 1e-5 (the per-particle maximum) and 4 max |a| it bounds every single star.  The binary
    members' own velocities are not compared: over their ~2^23 sub-steps a 1e-16 difference in
    phase grows to O(1e-2) of their orbital speed in FP64 itself."""
    n = 4096
    m, x, v = ics.plummer_kroupa_binaries(n, 31)
    ns = n - 2 * int(round(0.05 * n / 2.0))
    t = 2.0 ** -10
    out = {}
    for prec in ("fp64", "mixed"):
        f = F(m, x, v, precision=prec, eta=0.2)
        e0 = f.energy()["E"]
        f.step(t, 1)
        e1 = f.energy()["E"]
        xg, vg, _ = f.state()
        out[prec] = (xg, vg, abs((e1 - e0) / e0), f.stats()["max_depth_seen"])
        f.close()
    assert out["fp64"][3] == out["mixed"][3] >= 15, (out["fp64"][3], out["mixed"][3])
    assert out["mixed"][2] <= 2.0 * out["fp64"][2], (out["mixed"][2], out["fp64"][2])
    singles = np.arange(ns, dtype=np.int32)
    a0 = np.linalg.norm(oracle.acc(m, x, singles, np.arange(n, dtype=np.int32)), axis=1)
    A = 2.0 * np.percentile(a0, 99.0)
    dx = np.linalg.norm(out["mixed"][0][:ns] - out["fp64"][0][:ns], axis=1)
    dv = np.linalg.norm(out["mixed"][1][:ns] - out["fp64"][1][:ns], axis=1)
    assert p999(dx) < 0.5 * 2e-7 * A * t * t, (p999(dx), A)
    assert p999(dv) < 2e-7 * A * t, (p999(dv), A)
    amax = 4.0 * a0.max()
    assert dx.max() < 0.5 * 1e-5 * amax * t * t and dv.max() < 1e-5 * amax * t, (dx.max(), dv.max(), amax)


def test_plummer_64k_mixed_trajectory_matches_fp64():
    """Plummer N = 65536 (seed 2), two top-level steps of 2^-7 (t = 2^-6) in the mixed mode and
    in the FP64 mode on the GPU, compared particle by particle.

    Tolerance, from the arithmetic: the mixed Newtonian pass carries a relative error of
    0.7-1.4e-7 at the 99.9th percentile (at most 1e-5 per particle), and a kick or drift adds
    no error of its own (FP64, the oracle's roundings), so an acceleration error eps |a|
    held over the run moves v by eps |a| t and x by eps |a| t^2 / 2.  With eps = 2e-7 and
    |a| = 2 (above the 99th percentile of |a| in the sphere, 1.3) the 99.9th percentiles are
    bounded by 6.2e-9 (v) and 4.9e-11 (x); the 32 largest deviations are each bounded with
    eps = 1e-5 and 4 max(|a_i|, 2), |a_i| from the oracle at t = 0.  The two runs reach the
    same depth."""
    m, x, v = ics.workload("plummer_64k")
    n = m.size
    t = 2.0 * 2.0 ** -7
    out = {}
    for prec in ("fp64", "mixed"):
        f = F(m, x, v, precision=prec, eta=0.2)
        f.step(2.0 ** -7, 2)
        xg, vg, _ = f.state()
        out[prec] = (xg, vg, f.stats()["max_depth_seen"])
        f.close()
    assert out["fp64"][2] == out["mixed"][2]
    dx = np.linalg.norm(out["mixed"][0] - out["fp64"][0], axis=1)
    dv = np.linalg.norm(out["mixed"][1] - out["fp64"][1], axis=1)
    eps, A = 2e-7, 2.0
    assert p999(dx) < 0.5 * eps * A * t * t, p999(dx)
    assert p999(dv) < eps * A * t, p999(dv)
    top = np.argsort(np.maximum(dx / (t * t), dv / t))[-32:].astype(np.int32)
    a_top = np.linalg.norm(oracle.acc(m, x, top, np.arange(n, dtype=np.int32)), axis=1)
    bound_a = 1e-5 * 4.0 * np.maximum(a_top, A)
    assert np.all(dx[top] < 0.5 * bound_a * t * t), (dx[top].max(), a_top)
    assert np.all(dv[top] < bound_a * t), (dv[top].max(), a_top)


# ---------------------------------------------------------------------------------------
# the other full-size workloads, checked on sampled particles
# ---------------------------------------------------------------------------------------

def test_full_size_kroupa_binaries_262k_sampled():
    """Plummer N = 262144 with Kroupa masses and 5% hard binaries (seed 3): full mixed acc +
    gradient and time-step passes, 384 sampled particles (binary members included) against
    the oracle; the oracle computes every a_j for the sampled gradients."""
    m, x, v = ics.workload("plummer_kroupa_binaries_256k")
    n = m.size
    f = F(m, x, v, precision="mixed", eta=0.2)
    out = f.accel_gradient(None, None, eps_grad=2.0 ** -10)
    tau = cpu(f.timesteps())
    rng = np.random.default_rng(12)
    I = np.sort(np.concatenate([rng.choice(n - 13106, 256, replace=False),
                                n - 13106 + rng.choice(13106, 128, replace=False)])).astype(np.int32)
    A = np.arange(n, dtype=np.int32)
    a_all = oracle.acc(m, x, A, A)
    g_ref = oracle.grad(m, x, I, a_all[I], A, a_all)
    ea = rel(cpu(out["acc"])[I], a_all[I])
    eg = rel(cpu(out["grad"])[I], g_ref)
    et = rel(tau[I], oracle.timesteps_of(m, x, v, I, A, eta=0.2))
    assert p999(ea) < 1e-6 and p999(eg) < 1e-6, (p999(ea), p999(eg))
    assert p999(et) < 2e-6, p999(et)
    a = cpu(out["acc"])
    Ftot = (m[:, None] * a).sum(0)
    assert np.all(np.abs(Ftot) < 1e-9 * (m[:, None] * np.abs(a)).sum())
    f.close()


def test_full_size_plummer_1m_sampled_acc():
    """Plummer N = 1048576 (seed 5): the full mixed Newtonian pass on 256 sampled particles
    against the oracle, plus the vanishing total force over all particles."""
    m, x, v = ics.workload("plummer_1m")
    n = m.size
    f = F(m, x, v, precision="mixed")
    a = cpu(f.accel_gradient(None, None, want=("acc",))["acc"])
    rng = np.random.default_rng(13)
    I = np.sort(rng.choice(n, 256, replace=False)).astype(np.int32)
    ea = rel(a[I], oracle.acc(m, x, I, np.arange(n, dtype=np.int32)))
    assert p999(ea) < 1e-6 and ea.max() < 1e-5, (p999(ea), ea.max())
    Ftot = (m[:, None] * a).sum(0)
    assert np.all(np.abs(Ftot) < 1e-9 * (m[:, None] * np.abs(a)).sum())
    f.close()
