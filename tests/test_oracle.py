"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it checks.  None of them compares the oracle with
itself: the references are an independent Philox (Triton's interpreter), an
arbitrary-precision threshold computation, exact laws by enumeration written
from the paper's formulas, closed forms, and deterministic limits of the
dynamics that expose the neighbour geometry and the sign of the couplings.
"""
import json
import os
import subprocess
import sys

import mpmath
import numpy as np
import pytest
from scipy import optimize, stats

from oracle import exact

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


# ------------------------------------------------------------------ Philox

_TRITON_SCRIPT = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl

@triton.jit
def _k(out_ptr, c_ptr, seed, n: tl.constexpr):
    offs = tl.arange(0, n)
    c0 = tl.load(c_ptr + offs * 4 + 0)
    c1 = tl.load(c_ptr + offs * 4 + 1)
    c2 = tl.load(c_ptr + offs * 4 + 2)
    c3 = tl.load(c_ptr + offs * 4 + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + offs * 4 + 0, a)
    tl.store(out_ptr + offs * 4 + 1, b)
    tl.store(out_ptr + offs * 4 + 2, c)
    tl.store(out_ptr + offs * 4 + 3, d)

cases = json.loads(sys.stdin.read())
res = []
for seed, ctrs in cases:
    n = len(ctrs)
    flat = [((x + 2**31) % 2**32) - 2**31 for c in ctrs for x in c]
    cin = torch.tensor(flat, dtype=torch.int32)
    out = torch.zeros(4 * n, dtype=torch.int32)
    _k[(1,)](out, cin, seed, n=n)
    res.append([x & 0xffffffff for x in out.tolist()])
print(json.dumps(res))
"""


def test_philox_matches_independent_implementation(orc):
    """Philox4x32-10 (Salmon et al., SC'11) against Triton's own Philox run by
    its CPU interpreter: a third-party implementation of the same published
    algorithm, with the 64-bit seed split into (low, high) key words."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(11)
    cases = []
    for _ in range(4):
        seed = int(rng.integers(0, 2**63))
        ctrs = rng.integers(0, 2**32, size=(16, 4), dtype=np.uint64).tolist()
        ctrs[0] = [0, 0, 0, 0]
        cases.append([seed, ctrs])
    cases.append([0, [[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1],
                      [2**32 - 1] * 4, [5, 7, 9, 11], [0, 0, 1, 0], [3, 3, 3, 3],
                      [1, 2, 3, 4], [4, 3, 2, 1], [0, 2**31, 0, 0], [2**31, 0, 0, 0],
                      [9, 9, 9, 9], [10, 0, 0, 0], [11, 0, 0, 0], [12, 0, 0, 0]]])
    env = dict(os.environ, TRITON_INTERPRET="1")
    proc = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                          capture_output=True, text=True, env=env, timeout=600)
    if proc.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + proc.stderr[-300:])
    ref = json.loads(proc.stdout.strip().splitlines()[-1])
    for (seed, ctrs), want in zip(cases, ref):
        key = [seed & 0xffffffff, seed >> 32]
        got = [int(x) for c in ctrs for x in orc.philox4x32_10(c, key)]
        assert got == want


def test_philox_output_statistics(orc):
    """Bit balance and byte uniformity of the generator over consecutive block
    counters, as the per-site uniforms use them."""
    out = np.concatenate([orc.block_uniforms(0xC0FFEE, 5, w, 3, 0) for w in range(2048)])
    bits = ((out[:, None] >> np.arange(32)[None, :]) & 1).sum(axis=0)
    n = out.size
    z = (bits - n / 2) / np.sqrt(n / 4)
    assert np.abs(z).max() < 5.0
    hist = np.bincount((out & 0xFF).astype(np.int64), minlength=256)
    assert stats.chisquare(hist).pvalue > 1e-4
    top = np.bincount((out >> 24).astype(np.int64), minlength=256)
    assert stats.chisquare(top).pvalue > 1e-4


def test_block_uniform_transposition(orc):
    """Reading R5: r(32w + p) bit (31 - b) is bit p of the b-th Philox word of
    the block (counter (hs, w, lattice, c), outputs R[4c..4c+3])."""
    seed, hs, w, lat = 0x1234_5678_9ABC_DEF0, 17, 1234, 9
    key = [seed & 0xffffffff, seed >> 32]
    R = np.concatenate([orc.philox4x32_10([hs, w, lat, c], key) for c in range(8)])
    r = orc.block_uniforms(seed, hs, w, lat, 0)
    for p in (0, 1, 13, 31):
        v = 0
        for b in range(32):
            v |= int((int(R[b]) >> p) & 1) << (31 - b)
        assert int(r[p]) == v
    # the init domain is a disjoint stream
    assert not np.array_equal(r, orc.block_uniforms(seed, hs, w, lat, 1))


# -------------------------------------------------------------- thresholds

_QJ = [(1.0, 0.25), (0.5, 0.5), (1.0, 0.35), (0.6585, 0.6585), (3.0, 0.44), (0.05, 1.7),
       (2.5, 0.46), (0.0, 0.0), (0.0, 20.0), (20.0, 0.0), (-0.7, 0.3), (0.4, -1.1),
       (1e-9, 3e-10), (12.0, 5.0)]


@pytest.mark.parametrize("q,J", _QJ)
def test_thresholds_against_arbitrary_precision(orc, q, J):
    """P(+1) = e^{h}/(2 cosh h) (Algorithm 3, Eqs. leftTrans/rightTrans) with the
    field h = q s + J (2n - 2) of class k = 3[s=+1] + n: every integer threshold
    is within one unit of 2^32 p(h) computed with 60 significant digits."""
    T = orc.thresholds(q, J)
    mpmath.mp.dps = 60
    for s01 in (0, 1):
        for n in range(3):
            h = mpmath.mpf(q) * (2 * s01 - 1) + mpmath.mpf(J) * (2 * n - 2)
            p = mpmath.e ** h / (2 * mpmath.cosh(h))
            exact_scaled = p * mpmath.mpf(2) ** 32
            assert abs(int(T[3 * s01 + n]) - exact_scaled) <= 1, (s01, n)
            if h == 0:
                assert int(T[3 * s01 + n]) == 2 ** 31


@pytest.mark.parametrize("q,J", _QJ)
def test_threshold_spin_flip_complement(orc, q, J):
    """Reading R4: T(-h) = 2^32 - T(h), so the quantised chain keeps the exact
    +/- symmetry of the model; class k and class 5 - k carry opposite fields."""
    T = orc.thresholds(q, J).astype(np.int64)
    for k in range(6):
        h = q * (2 * (k // 3) - 1) + J * (2 * (k % 3) - 2)
        if h != 0:
            assert T[k] + T[5 - k] == 2 ** 32
    assert T.min() >= 1 and T.max() <= 2 ** 32 - 1


def test_thresholds_reject_non_finite(orc):
    for bad in (float("nan"), float("inf"), -float("inf")):
        with pytest.raises(ValueError):
            orc.thresholds(bad, 0.3)
        with pytest.raises(ValueError):
            orc.thresholds(0.3, bad)


def test_strict_comparison_on_ties(orc):
    """Algorithm 3 draws +1 when rand() < p (strict).  With a threshold table
    set equal to a site's own uniform the site must come out -1, and +1 when
    the threshold is one larger (reading R3)."""
    L, seed, lat, hs = 8, 99, 3, 6
    src = np.ones(L * L, dtype=np.int8)
    r = orc.block_uniforms(seed, hs, 1, lat, 0)          # sites 32..63
    for p_ in (0, 7, 31):
        u = 32 + p_
        for thr, want in ((int(r[p_]), -1), (int(r[p_]) + 1, 1)):
            T = np.full(6, thr, dtype=np.uint32)
            out = orc.halfstep(0, src, L, T, seed, lat, hs)
            assert out[u] == want


# ------------------------------------------------ geometry and couplings

def _single_plus(L, x):
    s = -np.ones(L * L, dtype=np.int8)
    s[x] = 1
    return s


@pytest.mark.parametrize("L,i0,j0", [(5, 1, 2), (7, 6, 0), (7, 0, 6), (33, 32, 5)])
def test_half_step_A_reads_down_and_left(orc, L, i0, j0):
    """Eq. urdl, left field: with q = 0 and J = 20 a site of tau can be +1 only
    when exactly one of sigma at x^down, x^left is +1 (field 0: a fair coin).
    A single + spin of sigma at x therefore randomises tau exactly at x^up
    = (i, j+1) and x^right = (i+1, j)."""
    T = orc.thresholds(0.0, 20.0)
    x = j0 * L + i0
    sig = _single_plus(L, x)
    hits = np.zeros(L * L, dtype=np.int64)
    for lat in range(200):
        tau = orc.halfstep(0, sig, L, T, seed=77, lattice_id=lat, hs=0)
        hits += tau > 0
    want = {((j0 + 1) % L) * L + i0, j0 * L + (i0 + 1) % L}
    assert set(np.nonzero(hits)[0].tolist()) == want
    for u in want:
        assert 60 < hits[u] < 140


@pytest.mark.parametrize("L,i0,j0", [(5, 1, 2), (7, 6, 0), (7, 0, 6), (33, 0, 0)])
def test_half_step_B_reads_up_and_right(orc, L, i0, j0):
    """Eq. urdl, right field: a single + spin of tau at y randomises sigma
    exactly at y^down = (i, j-1) and y^left = (i-1, j)."""
    T = orc.thresholds(0.0, 20.0)
    y = j0 * L + i0
    tau = _single_plus(L, y)
    hits = np.zeros(L * L, dtype=np.int64)
    for lat in range(200):
        sig = orc.halfstep(1, tau, L, T, seed=78, lattice_id=lat, hs=1)
        hits += sig > 0
    want = {((j0 - 1) % L) * L + i0, j0 * L + (i0 - 1) % L}
    assert set(np.nonzero(hits)[0].tolist()) == want


@pytest.mark.parametrize("half", [0, 1])
def test_self_coupling_copies_the_other_sublattice(orc, half):
    """The q (self-interaction) term of Eq. urdl with the ferromagnetic sign of
    reading R2: for J = 0, q = 20 each half-step copies the spin of the paired
    site (P = e^{20}/(2 cosh 20), one miss in 2^32); q = -20 copies it flipped."""
    L = 9
    rng = np.random.default_rng(3)
    src = rng.choice(np.array([-1, 1], dtype=np.int8), size=L * L)
    for q, sign in ((20.0, 1), (-20.0, -1)):
        T = orc.thresholds(q, 0.0)
        for lat in range(5):
            dst = orc.halfstep(half, src, L, T, seed=5, lattice_id=lat, hs=half)
            assert np.array_equal(dst, (sign * src).astype(np.int8))


def test_strong_J_aligns_with_neighbours(orc):
    """With J = 20, q = 0 an all + (all -) sublattice forces the other one to
    all + (all -): the field 2J of two agreeing neighbours dominates."""
    L = 6
    T = orc.thresholds(0.0, 20.0)
    for half in (0, 1):
        for v in (1, -1):
            src = np.full(L * L, v, dtype=np.int8)
            assert np.all(orc.halfstep(half, src, L, T, 1, 0, half) == v)


# -------------------------------------------------------- J = 0 closed form

def test_independent_spins_at_J0(orc):
    """J = 0 leaves every site an independent two-state chain that keeps its
    spin with probability a = T(q)/2^32 at each half-step.  From all +:
    E[sigma_t] = (2a-1)^(2t), E[tau_t] = (2a-1)^(2t-1), E[sigma_t tau_t] = 2a-1,
    all with binomial fluctuations."""
    L, q, M, n = 16, 0.3, 300, 3
    N = L * L
    a = int(orc.thresholds(q, 0.0)[3]) / 2 ** 32
    obs = np.zeros((M, n, 5), dtype=np.int64)
    for lat in range(M):
        s = np.ones(N, dtype=np.int8)
        t = np.ones(N, dtype=np.int8)
        obs[lat] = orc.run(s, t, L, q, 0.0, seed=21, lattice_id=lat, t0=0, n=n)
    for t in range(1, n + 1):
        for col, mean in ((0, (2 * a - 1) ** (2 * t)), (1, (2 * a - 1) ** (2 * t - 1)),
                          (2, 2 * a - 1)):
            x = obs[:, t - 1, col]
            var = N * (1 - mean ** 2)
            z = (x.mean() - N * mean) / np.sqrt(var / M)
            assert abs(z) < 5, (t, col, z)


# ------------------------------------------------------------ factorisation

def test_half_step_factorises_over_sites(orc):
    """Eq. fact / leftTrans: given sigma, the spins of tau are independent, each
    +1 with probability T[k_u]/2^32 (binomial test per site, 2x2 independence
    tests on neighbouring pairs)."""
    L, q, J, M = 5, 0.8, 0.4, 20000
    rng = np.random.default_rng(8)
    sig0 = rng.choice(np.array([-1, 1], dtype=np.int8), size=L * L)
    _, tau = orc.many_chains(L, q, J, seed=99, id0=0, M=M, init_sigma=sig0, n=1, want_tau=True)
    bits = ((tau[:, None] >> np.arange(L * L, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(np.int64)
    T = orc.thresholds(q, J)
    S = sig0.astype(np.int64)[None, :]
    k = exact.field_classes(S, L, "left")[0]
    p = T[k].astype(np.float64) / 2 ** 32
    z = (bits.sum(axis=0) - M * p) / np.sqrt(M * p * (1 - p))
    assert np.abs(z).max() < 5.0
    for a_, b_ in ((0, 1), (0, 5), (12, 13), (12, 17), (4, 0)):
        table = np.array([[np.sum((bits[:, a_] == x) & (bits[:, b_] == y)) for y in (0, 1)]
                          for x in (0, 1)])
        assert stats.chi2_contingency(table)[1] > 1e-4


# ------------------------------------------------------------ exact laws

@pytest.mark.parametrize("L", [2, 3])
@pytest.mark.parametrize("q,J", [(1.0, 0.25), (0.6585, 0.6585), (3.0, 0.44), (0.05, 1.7)])
def test_enumerated_stationary_law_is_the_closed_form(L, q, J):
    """The shaken kernel P^sq = P_A P_B enumerated from Eqs. leftTrans and
    rightTrans has stationary law pi_s(sigma) = Z_sigma / Z with
    Z_sigma = prod_u 2 cosh(<-h_u(sigma)) (Section 2)."""
    P = exact.shaken_kernel(L, q, J)
    assert np.allclose(P.sum(axis=1), 1.0, atol=1e-13)
    pi = exact.stationary(P)
    ref = exact.pi_s_closed_form(L, q, J)
    assert np.max(np.abs(pi - ref) / ref) < 1e-9


@pytest.mark.parametrize("q,J", [(1.0, 0.25), (0.6585, 0.6585)])
def test_pair_gibbs_measure_is_invariant(q, J):
    """pi_2(sigma, tau) proportional to e^{-H} of Eq. gs_ham2 is invariant for
    one full step of the alternate chain, and its sigma-marginal is pi_s."""
    L = 2
    pi2 = exact.pi_2(L, q, J)
    PA, PB = exact.half_step_kernels(L, q, J)
    # pair (sigma_t, tau_t): tau_t ~ P_A(sigma_{t-1}, .), sigma_t ~ P_B(tau_t, .)
    marg_sigma = pi2.sum(axis=1)
    new = (marg_sigma @ PA)[:, None] * PB          # new[tau, sigma]
    assert np.allclose(new.T, pi2, rtol=1e-10, atol=1e-15)
    assert np.allclose(marg_sigma, exact.pi_s_closed_form(L, q, J), rtol=1e-10)


@pytest.mark.parametrize("q,J", [(1.0, 0.25), (3.0, 0.44), (0.05, 1.7)])
def test_quantised_chain_stays_close_to_exact(orc, q, J):
    """Reading R3 changes each site probability by at most 2^-32, so the
    quantised chain's stationary law is within 1e-6 of pi_s in total variation."""
    L = 3
    pi_q = exact.stationary(exact.shaken_kernel(L, q, J, orc.thresholds(q, J)))
    assert 0.5 * np.abs(pi_q - exact.pi_s_closed_form(L, q, J)).sum() < 1e-6


def test_quantised_stationary_law_is_flip_symmetric(orc):
    """With the complement rule the quantised chain commutes with the global
    flip sigma -> -sigma, so its stationary law is exactly flip symmetric."""
    L, q, J = 3, 0.7, 0.55
    pi_q = exact.stationary(exact.shaken_kernel(L, q, J, orc.thresholds(q, J)))
    flipped = (2 ** 9 - 1) - np.arange(2 ** 9)
    assert np.allclose(pi_q, pi_q[flipped], rtol=1e-12, atol=0)


def _chi2_pvalue(counts, probs, min_expected=5.0):
    impossible = probs == 0
    assert counts[impossible].sum() == 0, "an outcome of probability zero occurred"
    counts, probs = counts[~impossible], probs[~impossible]
    exp_ = probs * counts.sum()
    order = np.argsort(exp_)
    small = exp_[order] < min_expected
    obs_big = counts[order][~small]
    exp_big = exp_[order][~small]
    if small.any():
        obs_big = np.append(obs_big, counts[order][small].sum())
        exp_big = np.append(exp_big, exp_[order][small].sum())
    return stats.chisquare(obs_big, exp_big * obs_big.sum() / exp_big.sum()).pvalue


def test_oracle_one_step_law_3x3(orc):
    """One step of the oracle from a fixed, asymmetric sigma on the 3x3 torus:
    the law of tau_1 is row sigma_0 of P_A and the law of sigma_1 is row
    sigma_0 of P^sq, both enumerated from the paper's formulas (chi-square)."""
    L, q, J, M = 3, 0.9, 0.45, 60000
    sig0 = np.array([1, 1, -1, 1, -1, -1, -1, 1, -1], dtype=np.int8)
    code0 = int(sum(1 << u for u in range(9) if sig0[u] > 0))
    T = orc.thresholds(q, J)
    PA, PB = exact.half_step_kernels(L, q, J, T)
    cs, ct = orc.many_chains(L, q, J, seed=4242, id0=0, M=M, init_sigma=sig0, n=1, want_tau=True)
    assert _chi2_pvalue(np.bincount(ct.astype(np.int64), minlength=512), PA[code0]) > 1e-4
    assert _chi2_pvalue(np.bincount(cs.astype(np.int64), minlength=512), (PA @ PB)[code0]) > 1e-4


def test_oracle_converges_to_stationary_law_3x3(orc):
    """Long-run law of the oracle on the 3x3 torus against the exact stationary
    vector of the quantised P^sq (chi-square over independent chains).  Half of
    the chains start from all +, half from all -, and the run length is chosen
    so the exact distance of that mixture to stationarity is below 1e-4."""
    L, M, q, J = 3, 40000, 0.5, 0.5
    T = orc.thresholds(q, J)
    P = exact.shaken_kernel(L, q, J, T)
    pi = exact.stationary(P)
    start = np.zeros(512)
    start[511] = start[0] = 0.5
    n, dist = 0, 1.0
    while dist > 1e-4:
        start = start @ P
        n += 1
        dist = 0.5 * np.abs(start - pi).sum()
        assert n < 400
    up = orc.many_chains(L, q, J, seed=7, id0=1000, M=M // 2, init_sigma=np.ones(9, np.int8), n=n)
    dn = orc.many_chains(L, q, J, seed=7, id0=1000 + M // 2, M=M // 2,
                         init_sigma=-np.ones(9, np.int8), n=n)
    cs = np.concatenate([up, dn])
    assert _chi2_pvalue(np.bincount(cs.astype(np.int64), minlength=512), pi) > 1e-4


@pytest.mark.parametrize("q,J", [(0.6585, 0.6585), (3.0, 0.44), (0.05, 1.7), (1.0, 0.25)])
def test_oracle_preserves_stationary_law_3x3(orc, q, J):
    """pi_s is invariant (Section 2): chains whose initial sigma is drawn from
    the exact stationary vector of the quantised P^sq still follow it after
    four oracle steps (chi-square).  The seeded draw of the initial states is
    an input; near the critical curve the 3x3 chain mixes too slowly for a
    fixed start."""
    L, M, n = 3, 40000, 4
    T = orc.thresholds(q, J)
    pi = exact.stationary(exact.shaken_kernel(L, q, J, T))
    rng = np.random.default_rng(int(1000 * q + 10 * J))
    draws = np.bincount(rng.choice(512, size=M, p=pi), minlength=512)
    finals, lat = [], 0
    for code in np.nonzero(draws)[0]:
        init = np.where((int(code) >> np.arange(9)) & 1, 1, -1).astype(np.int8)
        finals.append(orc.many_chains(L, q, J, seed=17, id0=lat, M=int(draws[code]),
                                      init_sigma=init, n=n))
        lat += int(draws[code])
    cs = np.concatenate(finals)
    assert _chi2_pvalue(np.bincount(cs.astype(np.int64), minlength=512), pi) > 1e-4


def test_oracle_pair_law_2x2(orc):
    """The pair (sigma_t, tau_t) at stationarity follows pi_2 (Section 2;
    Theorem 2.1 of the cited work rests on it): chains started from sigma
    drawn from pi_s (the sigma-marginal of pi_2) give pairs distributed as
    pi_2 after any number of steps; chi-square over the 256 pairs."""
    L, q, J, M, n = 2, 0.8, 0.5, 40000, 3
    pi2 = exact.pi_2(L, q, J)                      # [sigma, tau]
    rng = np.random.default_rng(5)
    draws = np.bincount(rng.choice(16, size=M, p=pi2.sum(axis=1)), minlength=16)
    cs_all, ct_all, lat = [], [], 0
    for code in np.nonzero(draws)[0]:
        init = np.where((int(code) >> np.arange(4)) & 1, 1, -1).astype(np.int8)
        cs, ct = orc.many_chains(L, q, J, seed=31, id0=lat, M=int(draws[code]),
                                 init_sigma=init, n=n, want_tau=True)
        cs_all.append(cs)
        ct_all.append(ct)
        lat += int(draws[code])
    cs, ct = np.concatenate(cs_all), np.concatenate(ct_all)
    counts = np.bincount((cs * 16 + ct).astype(np.int64), minlength=256)
    assert _chi2_pvalue(counts, pi2.reshape(-1)) > 1e-4


# ---------------------------------------------------- pathwise invariants

def test_monotone_coupling_and_coalescence(orc):
    """Section 3.2: the dynamics preserves the partial order, so the chains
    started from all + and all - with the same random numbers stay ordered
    site by site, and once equal they stay equal."""
    L, q, J = 8, 0.7, 0.3
    N = L * L
    top_s, top_t = np.ones(N, np.int8), np.ones(N, np.int8)
    bot_s, bot_t = -np.ones(N, np.int8), -np.ones(N, np.int8)
    met = None
    for t in range(300):
        orc.run(top_s, top_t, L, q, J, 5, 2, t, 1, want_obs=False)
        orc.run(bot_s, bot_t, L, q, J, 5, 2, t, 1, want_obs=False)
        assert np.all(bot_s <= top_s) and np.all(bot_t <= top_t)
        if met is None and np.array_equal(top_s, bot_s):
            met = t
        if met is not None:
            assert np.array_equal(top_s, bot_s)
    assert met is not None


def test_two_forms_of_the_pair_hamiltonian(orc):
    """Eq. gs_ham2 writes H two ways; the oracle's S_J (first form) equals
    sum_x tau_x (sigma_{x down} + sigma_{x left}) (second form) exactly."""
    rng = np.random.default_rng(12)
    for L in (2, 3, 7, 32):
        s = rng.choice(np.array([-1, 1], np.int8), size=(L, L))
        t = rng.choice(np.array([-1, 1], np.int8), size=(L, L))
        obs = orc.observables(s, t, L)
        S, Tt = s.astype(np.int64), t.astype(np.int64)
        down = np.roll(S, 1, axis=0)     # sigma at (i, j-1) seen from row j
        left = np.roll(S, 1, axis=1)     # sigma at (i-1, j)
        up_s = np.roll(S, -1, axis=0)
        right_s = np.roll(S, -1, axis=1)
        assert obs[0] == S.sum() and obs[1] == Tt.sum()
        assert obs[2] == (S * Tt).sum()
        assert obs[3] == (Tt * (down + left)).sum()
        assert obs[4] == (S * (up_s + right_s)).sum()


def test_row_restricted_half_step_matches_full(orc):
    """The row-band form of a half-step (used for sampled checks at full size)
    gives the same spins as the full sweep on those rows."""
    L = 40
    rng = np.random.default_rng(2)
    src = rng.choice(np.array([-1, 1], np.int8), size=L * L)
    T = orc.thresholds(0.9, 0.4)
    full = orc.halfstep(1, src, L, T, 3, 4, 11)
    part = orc.halfstep(1, src, L, T, 3, 4, 11, row0=13, row1=29)
    assert np.array_equal(full[13 * L:29 * L], part[13 * L:29 * L])


def test_random_initial_state(orc):
    """Reading R6: a random start has each spin + with probability 1/2,
    independently, and equals the MSB rule on the init stream."""
    L = 64
    s = orc.init_plane(L, orc.INIT_RANDOM, init_seed=2, lattice_id=0, plane_index=0)
    z = (np.sum(s > 0) - L * L / 2) / np.sqrt(L * L / 4)
    assert abs(z) < 5
    r = orc.block_uniforms(2, 0, 3, 0, 1)
    assert np.array_equal(s[96:128] > 0, r < 2 ** 31)
    t = orc.init_plane(L, orc.INIT_RANDOM, init_seed=2, lattice_id=0, plane_index=1)
    assert not np.array_equal(s, t)
    assert np.all(orc.init_plane(5, orc.INIT_ALL_UP) == 1)
    assert np.all(orc.init_plane(5, orc.INIT_ALL_DOWN) == -1)


# --------------------------------------------------------- critical curve

def test_critical_curve_printed_values():
    """Section 2 prints lim_{q->inf} J_c(q) = 0.4406867 and J_c(q) = q at 0.6585."""
    with open(os.path.join(HERE, "golden", "critical_curve.json")) as f:
        g = json.load(f)
    # the printed digits are truncated, so allow one unit of the last digit
    assert abs(float(exact.critical_J(40.0)) - g["q_to_infinity_limit"]) < 10.0 ** -g["limit_digits"]
    q_star = optimize.brentq(lambda q: exact.critical_J(q) - q, 0.1, 2.0, xtol=1e-14)
    assert abs(q_star - g["hexagonal_J_equals_q"]) < 10.0 ** -g["hexagonal_digits"]
    # the explicit critical condition of Eq. eqcrit holds along the curve
    for q in (0.1, 0.5, 1.0, 2.5):
        J = exact.critical_J(q)
        assert abs(2 * np.tanh(J) * np.tanh(q) + np.tanh(J) ** 2 - 1) < 1e-12


# ------------------------------------------------- diagonal correlations

def test_diagonal_correlation_sums(orc):
    """Section 3.3's SW-NE pair (0,0)-(l,l) and NW-SE pair (0,l)-(l,0),
    averaged over translations: exact values for patterns with known answers
    and, for random planes, agreement with an independent numpy computation by
    array rolls."""
    L = 12
    i, j = np.meshgrid(np.arange(L), np.arange(L))          # i: column, j: row
    lags = [0, 1, 2, 3, 5, 11]
    N = L * L
    ones = np.ones(N, np.int8)
    assert np.all(orc.diag_correlations(ones, L, lags) == N)
    board = np.where((i + j) % 2 == 0, 1, -1).astype(np.int8).ravel()
    assert np.all(orc.diag_correlations(board, L, lags) == N)
    cols = np.where(i % 2 == 0, 1, -1).astype(np.int8).ravel()    # depends on the column only
    got = orc.diag_correlations(cols, L, lags)
    want = np.array([N * (-1) ** l for l in lags] * 2)
    assert np.array_equal(got, want)
    rows_ = np.where(j % 3 == 0, 1, -1).astype(np.int8)       # depends on the row only
    got = orc.diag_correlations(rows_.ravel(), L, lags)
    for k, l in enumerate(lags):
        assert got[k] == np.sum(rows_ * np.roll(rows_, -l, axis=0))
        assert got[len(lags) + k] == np.sum(rows_ * np.roll(rows_, l, axis=0))
    rng = np.random.default_rng(1)
    for L2 in (7, 16):
        s = rng.choice(np.array([-1, 1], np.int8), size=(L2, L2))
        got = orc.diag_correlations(s.ravel(), L2, [1, 2, 4])
        S = s.astype(np.int64)
        for k, l in enumerate([1, 2, 4]):
            swne = np.roll(np.roll(S, -l, axis=0), -l, axis=1)   # s at (i+l, j+l)
            nwse = np.roll(np.roll(S, l, axis=0), -l, axis=1)    # s at (i+l, j-l)
            assert got[k] == np.sum(S * swne)
            assert got[3 + k] == np.sum(S * nwse)


# ----------------------------------------------- checkerboard heat bath (Section 3.2)

@pytest.mark.parametrize("J", [0.2, 0.4406867, 0.9, -0.5, 0.0])
def test_checkerboard_thresholds_against_arbitrary_precision(orc, J):
    """P(+1) = e^{h}/(2 cosh h), h = J (2n - 4) for n = 0..4 + neighbours."""
    T = orc.checkerboard_thresholds(J)
    mpmath.mp.dps = 60
    for n in range(5):
        h = mpmath.mpf(J) * (2 * n - 4)
        assert abs(int(T[n]) - mpmath.e ** h / (2 * mpmath.cosh(h)) * mpmath.mpf(2) ** 32) <= 1
        if h != 0:
            assert int(T[n]) + int(T[4 - n]) == 2 ** 32


@pytest.mark.parametrize("J", [0.3, 0.7])
def test_checkerboard_kernels_preserve_square_gibbs(J):
    """Theorem 2.2 of the cited work: each parity's heat-bath redraw leaves the
    square-lattice Gibbs measure invariant (2x2 torus, exact enumeration)."""
    pi = exact.square_gibbs(2, J)
    for parity in (0, 1):
        K = exact.checkerboard_kernel(2, J, parity)
        assert np.allclose(K.sum(axis=1), 1.0, atol=1e-13)
        assert np.max(np.abs(pi @ K - pi)) < 1e-14


def test_checkerboard_half_step_law_2x2(orc):
    """One oracle half-step from a fixed state against the row of the
    enumerated (quantised) kernel, for both parities (chi-square)."""
    L, J, M = 2, 0.5, 40000
    T = orc.checkerboard_thresholds(J)
    s0 = np.array([1, -1, -1, -1], dtype=np.int8)
    code0 = 1
    for parity in (0, 1):
        K = exact.checkerboard_kernel(L, J, parity, T)
        counts = np.zeros(16, dtype=np.int64)
        for lat in range(M):
            s = s0.copy()
            orc.checkerboard_halfstep(s, L, T, 11, lat, parity, parity)
            counts[int(np.sum((s > 0).astype(np.int64) << np.arange(4)))] += 1
        assert _chi2_pvalue(counts, K[code0]) > 1e-4


def test_checkerboard_preserves_gibbs_4x4(orc):
    """States drawn from the exact 4x4 square-lattice Gibbs measure stay
    Gibbs-distributed under the oracle's checkerboard steps: chi-square on the
    joint histogram of (magnetisation, energy)."""
    L, J, M, n = 4, 0.4, 30000, 3
    S = exact.spin_table(16)
    pi = exact.square_gibbs(L, J)
    Mag = S.sum(axis=1)
    up, right, _, _ = exact.neighbours(L)
    C = np.sum(S * (S[:, up] + S[:, right]), axis=1)
    key = (Mag + 16) * 100 + (C + 40)
    keys, inv = np.unique(key, return_inverse=True)
    probs = np.bincount(inv, weights=pi, minlength=keys.size)
    rng = np.random.default_rng(44)
    codes = rng.choice(2 ** 16, size=M, p=pi)
    counts = np.zeros(keys.size, dtype=np.int64)
    for k, code in enumerate(codes):
        s = np.where((int(code) >> np.arange(16)) & 1, 1, -1).astype(np.int8)
        obs = orc.checkerboard_run(s, L, J, 5, k, 0, n)
        kk = (obs[-1, 0] + 16) * 100 + (obs[-1, 1] + 40)
        counts[np.searchsorted(keys, kk)] += 1
    assert _chi2_pvalue(counts, probs) > 1e-4


def test_checkerboard_updates_one_parity_and_follows_strong_coupling(orc):
    """A half-step changes only the sites of its parity; with J = 20 a site
    with 3 or 4 + neighbours becomes +, with 0 or 1 becomes -."""
    L = 8
    T = orc.checkerboard_thresholds(20.0)
    rng = np.random.default_rng(3)
    s = rng.choice(np.array([-1, 1], np.int8), size=L * L)
    for parity in (0, 1):
        before = s.copy()
        orc.checkerboard_halfstep(s, L, T, 1, 0, 4 + parity, parity)
        j, i = np.divmod(np.arange(L * L), L)
        other = ((i + j) % 2) != parity
        assert np.array_equal(s[other], before[other])
        up, right, down, left = exact.neighbours(L)
        n = (before[up] > 0).astype(int) + (before[down] > 0) + (before[left] > 0) + (before[right] > 0)
        mine = ~other
        assert np.all(s[mine & (n >= 3)] == 1) and np.all(s[mine & (n <= 1)] == -1)


# ---- coupling from the past (Propp-Wilson, Section 3.2)

def _quantised_checkerboard_step(L, J, T5):
    return exact.checkerboard_kernel(L, J, 0, T5) @ exact.checkerboard_kernel(L, J, 1, T5)


@pytest.mark.parametrize("L,q,J", [(2, 0.5, 0.8), (2, 0.6585, 0.6585), (3, 1.0, 0.4)])
def test_cftp_samples_follow_the_stationary_law(orc, L, q, J):
    """Propp-Wilson returns exact draws from the stationary law of the
    quantised shaken chain (its stationary vector computed by enumeration);
    every attempt coalesces well before the cap."""
    M = 20000 if L == 2 else 30000
    codes, ks = orc.cftp_many(orc.SHAKEN, L, q, J, seed=77, id0=0, M=M, k_max=16)
    assert np.all(ks >= 0)
    pi = exact.stationary(exact.shaken_kernel(L, q, J, orc.thresholds(q, J)))
    counts = np.bincount(codes.astype(np.int64), minlength=2 ** (L * L))
    assert _chi2_pvalue(counts, pi) > 1e-4


def test_cftp_reuses_the_randomness_of_each_time(orc):
    """Starting further in the past changes nothing once an attempt has
    coalesced: the time-0 state from -2^(k+3) equals the one from -2^k (the
    step from -s to -s+1 always uses forward step index s - 1)."""
    L, q, J = 32, 0.8, 0.35
    k, s = orc.cftp(orc.SHAKEN, L, q, J, 5, 3, k_max=14)
    assert k >= 0
    for start in (2 ** k, 2 ** (k + 3)):
        top_s, top_t = np.ones(L * L, np.int8), np.ones(L * L, np.int8)
        bot_s, bot_t = -np.ones(L * L, np.int8), -np.ones(L * L, np.int8)
        for sidx in range(start, 0, -1):
            orc.run(top_s, top_t, L, q, J, 5, 3, sidx - 1, 1, want_obs=False)
            orc.run(bot_s, bot_t, L, q, J, 5, 3, sidx - 1, 1, want_obs=False)
        assert np.array_equal(top_s, s) and np.array_equal(bot_s, s)
    if k > 0:   # the attempt before the successful one had not coalesced
        top_s, top_t = np.ones(L * L, np.int8), np.ones(L * L, np.int8)
        bot_s, bot_t = -np.ones(L * L, np.int8), -np.ones(L * L, np.int8)
        for sidx in range(2 ** (k - 1), 0, -1):
            orc.run(top_s, top_t, L, q, J, 5, 3, sidx - 1, 1, want_obs=False)
            orc.run(bot_s, bot_t, L, q, J, 5, 3, sidx - 1, 1, want_obs=False)
        assert not np.array_equal(top_s, bot_s)


def test_cftp_checkerboard_follows_the_quantised_gibbs_law_2x2(orc):
    L, J, M = 2, 0.6, 20000
    T5 = orc.checkerboard_thresholds(J)
    pi = exact.stationary(_quantised_checkerboard_step(L, J, T5))
    assert np.max(np.abs(pi - exact.square_gibbs(L, J))) < 1e-8
    codes, ks = orc.cftp_many(orc.CHECKERBOARD, L, 0.0, J, seed=31, id0=0, M=M, k_max=16)
    assert np.all(ks >= 0)
    assert _chi2_pvalue(np.bincount(codes.astype(np.int64), minlength=16), pi) > 1e-4


def test_cftp_checkerboard_4x4_magnetisation_energy_law(orc):
    """Perfect samples of the 4x4 checkerboard chain against the exact Gibbs
    law of (magnetisation, energy) near the critical coupling."""
    L, J, M = 4, 0.44, 12000
    S = exact.spin_table(16)
    pi = exact.square_gibbs(L, J)
    up, right, _, _ = exact.neighbours(L)
    key = (S.sum(axis=1) + 16) * 100 + (np.sum(S * (S[:, up] + S[:, right]), axis=1) + 40)
    keys, inv = np.unique(key, return_inverse=True)
    probs = np.bincount(inv, weights=pi, minlength=keys.size)
    codes, ks = orc.cftp_many(orc.CHECKERBOARD, L, 0.0, J, seed=8, id0=0, M=M, k_max=18)
    assert np.all(ks >= 0)
    counts = np.bincount(inv[codes.astype(np.int64)], minlength=keys.size)
    assert _chi2_pvalue(counts, probs) > 1e-4


def test_exact_diagonal_correlations_order_theorem_2_4(orc):
    """Section 3.3 (Theorem 2.4 of the cited work): under the stationary law
    pi_s the SW-NE correlation E[s_(0,0) s_(1,1)] lies below the NW-SE one
    E[s_(0,1) s_(1,0)] for small q, and the two meet as q grows.  Checked on
    the exact closed-form law of the 4x4 torus (65536 states), with the
    per-state sums taken from the oracle's diagonal-correlation routine."""
    L, N = 4, 16
    S = exact.spin_table(N)
    sums = np.array([orc.diag_correlations(S[c].astype(np.int8), L, [1]) for c in range(2 ** N)],
                    dtype=np.float64) / N        # columns: SW-NE, NW-SE
    gaps = []
    for q in (0.05, 0.2, 0.5, 1.0, 2.0, 3.0):
        pi = exact.pi_s_closed_form(L, q, 0.7)
        swne, nwse = pi @ sums[:, 0], pi @ sums[:, 1]
        gaps.append(nwse - swne)
    assert gaps[0] > 0.3 and all(g > 0 for g in gaps), gaps
    assert all(a > b for a, b in zip(gaps, gaps[1:])), gaps    # the gap closes as q grows
    assert gaps[-1] < 1e-2
