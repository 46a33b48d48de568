"""Pins of the FP64 oracle against facts that do not come from the oracle:
hand-worked examples, closed forms, textbook special cases, invariants of
the method and brute force on tiny inputs.  CPU only."""
import math

import numpy as np
import pytest

import spamm_inputs as gen
from oracle import oracle as O
from tests.golden_io import read_worked_examples


def _padded(A, b):
    n = A.shape[0]
    d = O.depth(n, b)
    npad = b << d
    P = np.zeros((npad, npad))
    P[:n, :n] = A.astype(np.float64)
    return P, d


def _leaf_norm2(A, b):
    """Leaf squared norms straight from numpy (independent of the oracle)."""
    P, d = _padded(A, b)
    nb = 1 << d
    return (P * P).reshape(nb, b, nb, b).sum(axis=(1, 3))


def _as_set(tr):
    return set(map(tuple, np.asarray(tr).tolist()))


# ------------------------------------------------------------- Eq. (depth)

@pytest.mark.parametrize("n,b,d", [(1000, 16, 6), (1024, 16, 6), (7500, 16, 9),
                                   (16384, 16, 10), (16384, 128, 7), (1, 16, 0),
                                   (16, 16, 0), (17, 16, 1), (8192, 16, 9)])
def test_depth_closed_form(n, b, d):
    assert O.depth(n, b) == d
    if n > b:   # the paper's formula itself, evaluated in floating point
        assert math.ceil(math.log(n / b) / math.log(2)) == d


# ------------------------------------------------------------- Eq. (norm)

@pytest.mark.parametrize("n,b", [(40, 4), (64, 16), (100, 16), (33, 8)])
def test_pyramid_matches_block_sums(n, b):
    A = gen.exp_decay_nonsym(n, 0.8, seed=3)
    pyr = O.pyramid(A, b)
    P, d = _padded(A, b)
    for t in range(d + 1):
        w = 1 << t
        s = (b << d) // w
        ref = (P * P).reshape(w, s, w, s).sum(axis=(1, 3))
        np.testing.assert_allclose(O.tier(pyr, t), ref, rtol=1e-13, atol=0)
    assert pyr[0] == pytest.approx(np.linalg.norm(A.astype(np.float64)) ** 2, rel=1e-13)


def test_parent_never_below_child():
    A = gen.water_like(20, 5)  # n = 100
    pyr = O.pyramid(A, 4)
    d = O.depth(100, 4)
    for t in range(d):
        par = O.tier(pyr, t)
        ch = O.tier(pyr, t + 1)
        w = 1 << t
        for di in range(2):
            for dj in range(2):
                assert np.all(par >= ch[di::2, dj::2][:w, :w])


# ----------------------------------------------------- hand-worked golden

def test_worked_examples():
    mats, cases = read_worked_examples()
    A = mats["A"]
    assert cases
    for case in cases:
        r = O.multiply(A, A, case["b"], case["tau"])
        assert sorted(_as_set(r.triples)) == case["triples"], case["name"]
        np.testing.assert_array_equal(r.C, case["C"], err_msg=case["name"])
        if "cand" in case:
            assert list(r.cand) == case["cand"]
            assert list(r.kept) == case["kept"]
        d = O.depth(4, case["b"])
        pa = O.pyramid(A, case["b"])
        assert _as_set(O.cull_linkless(pa, pa, d, case["tau"])) == set(case["triples"])


# ------------------------------------------------------------- tau = 0

@pytest.mark.parametrize("n,b", [(50, 8), (64, 16), (37, 4), (100, 32), (16, 16), (5, 16)])
def test_tau0_is_dense_product(n, b):
    A = gen.uniform_dense(n, seed=1, symmetric=False)
    B = gen.exp_decay_nonsym(n, 0.9, seed=2)
    r = O.multiply(A, B, b, 0.0)
    E = A.astype(np.float64) @ B.astype(np.float64)
    assert np.abs(r.C - E).max() <= 1e-13 * np.abs(E).max()
    nbr = -(-n // b)
    # every non-padding leaf is non-zero here, so all nbr^3 triples survive
    assert len(r.triples) == nbr ** 3


def test_transpose_is_not_confused():
    n, b = 48, 8
    A = gen.exp_decay_nonsym(n, 0.7, seed=5)
    B = gen.uniform_dense(n, seed=6, symmetric=False)
    r1 = O.multiply(A, B, b, 0.0).C
    r2 = O.multiply(B.T.copy(), A.T.copy(), b, 0.0).C
    np.testing.assert_allclose(r1, r2.T, rtol=0, atol=1e-12)
    assert np.abs(r1 - r1.T).max() > 1e-3


# --------------------------------------- flat (Algorithm 1) == recursive

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_linkless_equals_recursive(seed):
    rng = np.random.default_rng(seed)
    for n, b in [(64, 4), (96, 8), (128, 16), (20, 2)]:
        A = gen.exp_decay_nonsym(n, float(rng.uniform(0.5, 0.95)), seed=seed)
        B = gen.water_like(4, n // 4, seed=seed)[:n, :n].copy() if n % 4 == 0 else A
        pa, pb = O.pyramid(A, b), O.pyramid(B, b)
        d = O.depth(n, b)
        for tau in [0.0] + list(10.0 ** rng.uniform(-8, 0, size=6)):
            rec = _as_set(O.cull_recursive(pa, pb, d, tau)[0])
            flat = _as_set(O.cull_linkless(pa, pb, d, tau))
            assert rec == flat


def test_brute_force_tiny():
    """Every leaf triple enumerated directly with numpy norms."""
    rng = np.random.default_rng(7)
    for n, b in [(8, 2), (12, 4), (16, 2), (9, 4)]:
        A = gen.exp_decay_nonsym(n, 0.6, seed=11)
        B = gen.exp_decay_nonsym(n, 0.5, seed=12)
        na, nb2 = _leaf_norm2(A, b), _leaf_norm2(B, b)
        w = na.shape[0]
        pa, pb = O.pyramid(A, b), O.pyramid(B, b)
        d = O.depth(n, b)
        for tau in 10.0 ** rng.uniform(-4, 0.5, size=8):
            want = {(i, k, j) for i in range(w) for k in range(w) for j in range(w)
                    if na[i, k] > 0 and nb2[k, j] > 0
                    and math.sqrt(na[i, k]) * math.sqrt(nb2[k, j]) >= tau * (1 + 1e-12)}
            maybe = {(i, k, j) for i in range(w) for k in range(w) for j in range(w)
                     if na[i, k] > 0 and nb2[k, j] > 0
                     and abs(math.sqrt(na[i, k] * nb2[k, j]) - tau) <= 1e-12 * tau}
            got = _as_set(O.cull_recursive(pa, pb, d, tau)[0])
            assert want <= got <= want | maybe
            # and the numeric part: each C block is the plain sum over kept K
            r = O.multiply(A, B, b, tau)
            P, _ = _padded(A, b)
            Q, _ = _padded(B, b)
            Cref = np.zeros_like(P)
            for (i, k, j) in got:
                Cref[i*b:(i+1)*b, j*b:(j+1)*b] += P[i*b:(i+1)*b, k*b:(k+1)*b] @ \
                    Q[k*b:(k+1)*b, j*b:(j+1)*b]
            np.testing.assert_allclose(r.C, Cref[:n, :n], rtol=1e-13, atol=1e-15)


# ------------------------------------------------------------ invariants

def test_monotone_nesting():
    A = gen.exp_decay(128, 0.85, seed=4)
    pa = O.pyramid(A, 8)
    d = O.depth(128, 8)
    prev = None
    for tau in [0, 1e-8, 1e-6, 1e-4, 1e-3, 1e-2, 1e-1, 1, 10]:
        s = _as_set(O.cull_recursive(pa, pa, d, tau)[0])
        if prev is not None:
            assert s <= prev
        prev = s


def test_tau_above_root_product():
    A = gen.exp_decay(64, 0.9, seed=1)
    B = gen.uniform_dense(64, seed=2)
    root = np.linalg.norm(A.astype(np.float64)) * np.linalg.norm(B.astype(np.float64))
    C0 = gen.uniform_dense(64, seed=3).astype(np.float64)
    r = O.multiply(A, B, 16, root * 1.0001, alpha=2.0, beta=-0.5, C=C0)
    assert len(r.triples) == 0
    np.testing.assert_array_equal(r.C, -0.5 * C0)
    r2 = O.multiply(A, B, 16, root * 0.9999)
    assert r2.kept[0] == 1                  # the root product itself survives
    na, nb2 = np.sqrt(_leaf_norm2(A, 16)), np.sqrt(_leaf_norm2(B, 16))
    best = max(na[i, k] * nb2[k, j] for i in range(4) for k in range(4) for j in range(4))
    assert len(O.multiply(A, B, 16, best * 0.9999).triples) >= 1
    assert len(O.multiply(A, B, 16, best * 1.0001).triples) == 0


def test_alpha_beta_epilogue():
    n = 40
    A = gen.exp_decay(n, 0.8, seed=1)
    C0 = gen.uniform_dense(n, seed=9, symmetric=False).astype(np.float64)
    base = O.multiply(A, A, 8, 1e-3).C
    r = O.multiply(A, A, 8, 1e-3, alpha=-1.5, beta=0.25, C=C0).C
    np.testing.assert_allclose(r, -1.5 * base + 0.25 * C0, rtol=1e-14, atol=1e-14)
    Cnan = np.full((n, n), np.nan)
    r0 = O.multiply(A, A, 8, 1e-3, alpha=1.0, beta=0.0, C=Cnan).C
    np.testing.assert_array_equal(r0, base)   # beta = 0: C is not read


@pytest.mark.parametrize("n,b,lam", [(128, 8, 0.85), (100, 16, 0.9), (96, 4, 0.7)])
def test_error_bound(n, b, lam):
    """||AB - C_tau||_F <= sum over culled leaf pairs of ||A_IK|| ||B_KJ||
    (triangle inequality and Frobenius submultiplicativity), which is
    < N_culled * tau."""
    A = gen.exp_decay_nonsym(n, lam, seed=21)
    B = gen.exp_decay_nonsym(n, lam, seed=22)
    E = A.astype(np.float64) @ B.astype(np.float64)
    na, nb2 = np.sqrt(_leaf_norm2(A, b)), np.sqrt(_leaf_norm2(B, b))
    w = na.shape[0]
    full = {(i, k, j) for i in range(w) for k in range(w) for j in range(w)
            if na[i, k] > 0 and nb2[k, j] > 0}
    for tau in [1e-6, 1e-4, 1e-2, 1e-1]:
        r = O.multiply(A, B, b, tau)
        kept = _as_set(r.triples)
        culled = full - kept
        bound = sum(na[i, k] * nb2[k, j] for (i, k, j) in culled)
        err = np.linalg.norm(E - r.C)
        assert err <= bound * (1 + 1e-12) + 1e-14
        assert bound <= len(culled) * tau * (1 + 1e-12)
        if not culled:
            assert err <= 1e-13 * np.abs(E).max()


def test_identity_special_case():
    """A = I: C_IJ = B_IJ exactly when sqrt(#diagonal ones in leaf I) *
    ||B_IJ|| >= tau, else 0."""
    n, b = 72, 16          # ragged: the last leaf holds 8 ones
    I = np.eye(n, dtype=np.float32)
    B = gen.exp_decay_nonsym(n, 0.8, seed=5)
    nbB = np.sqrt(_leaf_norm2(B, b))
    w = nbB.shape[0]
    for tau in [1e-6, 1e-3, 0.05, 0.5, 2.0]:
        r = O.multiply(I, B, b, tau)
        for bi in range(w):
            ones = max(0, min(n, (bi + 1) * b) - bi * b)
            for bj in range(w):
                blk = r.C[bi*b:(bi+1)*b, bj*b:(bj+1)*b]
                ref = B[bi*b:(bi+1)*b, bj*b:(bj+1)*b].astype(np.float64)
                keep = ones > 0 and nbB[bi, bj] > 0 and math.sqrt(ones) * nbB[bi, bj] >= tau
                np.testing.assert_array_equal(blk, ref if keep else 0 * ref)


def test_block_diagonal_exact():
    n, b = 64, 16
    rng = np.random.default_rng(3)
    A = np.zeros((n, n), dtype=np.float32)
    B = np.zeros((n, n), dtype=np.float32)
    for q in range(n // b):
        s = slice(q * b, (q + 1) * b)
        A[s, s] = rng.uniform(-1, 1, (b, b))
        B[s, s] = rng.uniform(-1, 1, (b, b))
    na, nb2 = np.sqrt(_leaf_norm2(A, b)), np.sqrt(_leaf_norm2(B, b))
    tau = 0.99 * min(na[q, q] * nb2[q, q] for q in range(n // b))
    r = O.multiply(A, B, b, tau)
    E = A.astype(np.float64) @ B.astype(np.float64)
    assert np.abs(r.C - E).max() <= 1e-14
    assert _as_set(r.triples) == {(q, q, q) for q in range(n // b)}


def test_algebraic_pm1_counts_are_sign_free():
    """|s_ij| = 1 makes every leaf norm independent of the signs, so the kept
    set does not depend on the seed and equals that of the all-positive
    magnitude matrix 1 / (|i-j|^2 + 1)."""
    n, b = 256, 16
    i = np.arange(n)
    M = (1.0 / ((i[:, None] - i[None, :]) ** 2 + 1.0)).astype(np.float32)
    d = O.depth(n, b)
    pm = O.pyramid(M, b)
    for tau in [1e-5, 1e-4, 1e-3]:
        ref = _as_set(O.cull_recursive(pm, pm, d, tau)[0])
        for seed in (0, 1):
            A = gen.algebraic_decay(n, seed=seed)
            pa = O.pyramid(A, b)
            assert _as_set(O.cull_recursive(pa, pa, d, tau)[0]) == ref


# ------------------------------------------------ Morton, Sec. III.D.1-2

def test_morton_hand_values():
    # l = sum_m i_m 2^(2m+1) + j_m 2^(2m)
    assert O.morton(0, 0) == 0
    assert O.morton(0, 1) == 1
    assert O.morton(1, 0) == 2
    assert O.morton(1, 1) == 3
    assert O.morton(2, 1) == 0b1001
    assert O.morton(3, 5) == 0b11011       # i bits 0,1 -> 1,3; j bits 0,2 -> 0,4
    assert O.morton(0xFFFF, 0) == int("10" * 16, 2)


def test_morton_tree_and_masks():
    rng = np.random.default_rng(0)
    for _ in range(200):
        i, k, j = (int(x) for x in rng.integers(0, 1 << 20, size=3))
        l = O.morton(i, j)
        assert O.morton_decode(l) == (i, j)
        for a in range(2):
            for c in range(2):   # a child appends two digits: parent * 4 + quadrant
                assert O.morton(2 * i + a, 2 * j + c) == 4 * l + 2 * a + c
        lA, lB = O.morton(i, k), O.morton(k, j)
        assert O.k_key_A(lA) == O.k_key_B(lB)            # same k digits
        assert O.convolve(lA, lB) == O.morton(i, j)      # Eq. (convolution)
        k2 = int(rng.integers(0, 1 << 20))
        if k2 != k:
            assert O.k_key_A(lA) != O.k_key_B(O.morton(k2, j))


# --------------------------------------------------- sampled blocks agree

def test_blocks_match_full_oracle():
    n, b = 200, 16
    A = gen.water_like(8, 25, seed=2)
    for tau in [0.0, 1e-3, 1e-1]:
        r = O.multiply(A, A, b, tau)
        ij = [(0, 0), (3, 7), (12, 12), (12, 0), (5, 9)]
        acc, _ = O.blocks(A, A, b, tau, ij)
        for q, (I, J) in enumerate(ij):
            blk = r.C[I*b:min(n, (I+1)*b), J*b:min(n, (J+1)*b)]
            np.testing.assert_allclose(acc[q][:blk.shape[0], :blk.shape[1]], blk,
                                       rtol=1e-13, atol=1e-15)


# ------------------------------------------- sub-leaf cull along k (R14)

def test_sliced_with_one_slice_per_leaf_is_plain_spamm():
    A = gen.exp_decay(100, 0.8, seed=1)
    for b, tau in [(16, 1e-3), (8, 1e-5), (32, 1e-2)]:
        C, m, kept, tested = O.multiply_sliced(A, A, b, b, tau)
        ref = O.multiply(A, A, b, tau)
        assert np.array_equal(C, ref.C)
        assert m == kept == tested == len(ref.triples)


def test_sliced_at_tau_zero_is_the_dense_product():
    A = gen.uniform_dense(70, seed=3, symmetric=False)
    B = gen.exp_decay_nonsym(70, 0.9, seed=4)
    C, m, kept, tested = O.multiply_sliced(A, B, 16, 4, 0.0)
    exact = A.astype(np.float64) @ B.astype(np.float64)
    assert np.abs(C - exact).max() <= 1e-12 * np.abs(exact).max()


def test_sliced_zero_panels_are_null_and_cost_no_accuracy():
    """Every leaf's k-columns 2, 3 (of 4) are zero in A: slice 1 of every
    leaf product has a zero panel, is dropped even at tau = 0 (R3), and the
    product is still exact."""
    n, b, g = 48, 4, 2
    A = gen.uniform_dense(n, seed=5, symmetric=False)
    A[:, np.arange(n) % 4 >= 2] = 0.0
    B = gen.uniform_dense(n, seed=6, symmetric=False)
    C, m, kept, tested = O.multiply_sliced(A, B, b, g, 0.0)
    assert tested == 2 * m and kept == m
    exact = A.astype(np.float64) @ B.astype(np.float64)
    assert np.abs(C - exact).max() <= 1e-12 * np.abs(exact).max()


@pytest.mark.parametrize("b,g,tau", [(16, 4, 1e-3), (16, 8, 3e-4), (32, 16, 1e-3)])
def test_sliced_error_bound_and_monotone(b, g, tau):
    """Each dropped slice product has norm below tau (Frobenius
    submultiplicativity), so ||C_leaf - C_sliced||_F < dropped * tau; fewer
    slices survive a larger tau."""
    A = gen.exp_decay(120, 0.85, seed=7)
    plain = O.multiply(A, A, b, tau).C
    C, m, kept, tested = O.multiply_sliced(A, A, b, g, tau)
    assert kept <= tested == m * (b // g)
    err = np.linalg.norm(plain - C)
    assert err <= (tested - kept) * tau * (1 + 1e-12)
    _, _, kept2, _ = O.multiply_sliced(A, A, b, g, tau * 3)
    assert kept2 <= kept


# ----------------------------------------- sparsification (Sec. II.D, R15)

def _norm2(A):
    return float((A.astype(np.float64) ** 2).sum())


def test_sparsify_at_the_consistent_tolerance_changes_no_product():
    """With epsilon = tau / max(||A||_F, ||B||_F), a dropped leaf's product
    with any leaf of the other operand is below tau (a leaf's norm never
    exceeds the whole matrix's), so the SpAMM product of the sparsified
    operands keeps the same leaf triples and gives the same C."""
    A = gen.exp_decay(160, 0.8, seed=2)
    B = gen.exp_decay_nonsym(160, 0.85, seed=3)
    for b, tau in [(8, 1e-4), (16, 1e-6), (16, 1e-2)]:
        m2 = max(_norm2(A), _norm2(B))
        As, na = O.sparsify(A, b, tau, m2)
        Bs, nb = O.sparsify(B, b, tau, m2)
        assert na < (160 // b) ** 2 or tau < 1e-5
        ref = O.multiply(A, B, b, tau)
        got = O.multiply(As, Bs, b, tau)
        assert np.array_equal(got.C, ref.C)
        assert sorted(map(tuple, got.triples)) == sorted(map(tuple, ref.triples))


def test_sparsify_drops_exactly_the_small_and_zero_leaves():
    n, b = 64, 8
    A = gen.uniform_dense(n, seed=9, symmetric=False)
    A[:8, 8:16] = 0.0                                   # a zero leaf
    A[16:24, :8] *= 1e-6                                # a small leaf
    As, m = O.sparsify(A, b, 1e-3, 1.0)
    assert m == 64 - 2
    assert not As[:8, 8:16].any() and not As[16:24, :8].any()
    mask = np.ones((n, n), bool)
    mask[:8, 8:16] = mask[16:24, :8] = False
    assert np.array_equal(As[mask], A[mask])
    # tau = 0 keeps every non-zero leaf
    As0, m0 = O.sparsify(A, b, 0.0, 1.0)
    assert m0 == 63 and np.array_equal(As0, A)


def test_sparsify_error_bound():
    """||A - A_s||_F^2 = sum of the dropped leaves' norms^2 < dropped *
    tau^2 / norm2_max."""
    A = gen.exp_decay(200, 0.85, seed=4)
    b, tau = 8, 3e-3
    m2 = _norm2(A)
    As, m = O.sparsify(A, b, tau, m2)
    dropped = (200 // b) ** 2 - m
    err2 = _norm2(A - As)
    assert dropped > 0 and err2 < dropped * tau * tau / m2


# ------------------------------------- precision chosen by norm (R16)

def test_round_sig_hand_values():
    """Rounding to p significant bits: halfway cases go to even (or away
    from zero), values already on the p-bit grid are fixed points."""
    u = 2.0 ** -11
    assert O.round_sig(1 + u, 11) == 1.0                      # tie, to even
    assert O.round_sig(1 + u, 11, ties_away=True) == 1 + 2 * u
    assert O.round_sig(1 + 3 * u, 11) == 1 + 4 * u            # tie, to even
    assert O.round_sig(1 + 1.5 * u, 11) == 1 + 2 * u          # above the tie
    assert O.round_sig(-(1 + u), 11, ties_away=True) == -(1 + 2 * u)
    assert O.round_sig(2047.0, 11) == 2047.0                  # 11 bits exactly
    assert O.round_sig(4095.0, 11) == 4096.0                  # carries into the exponent
    assert O.round_sig(0.0, 8) == 0.0
    assert O.round_sig(3.0 * 2.0 ** -200, 2) == 3.0 * 2.0 ** -200
    assert O.round_sig(math.pi, 53) == math.pi


def test_round_sig_matches_ieee_half_and_bfloat16():
    """p = 11 is IEEE half precision's significand and p = 8 bfloat16's:
    inside their normal ranges the oracle's rounding equals numpy's float16
    conversion and torch's bfloat16 conversion (both round to nearest
    even), computed independently of the oracle."""
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(4000) * 10.0 ** rng.uniform(-4, 4, 4000)).astype(np.float32)
    x = np.concatenate([x, np.float32(1.0) + np.float32(2.0 ** -11) * np.arange(-40, 40,
                                                                               dtype=np.float32)])
    x = x[(np.abs(x) >= 2.0 ** -14) & (np.abs(x) <= 60000.0)]    # float16's normal range
    h = x.astype(np.float16).astype(np.float64)
    got = np.array([O.round_sig(float(v), 11) for v in x])
    assert np.array_equal(got, h)
    torch = pytest.importorskip("torch")
    bf = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got8 = np.array([O.round_sig(float(v), 8) for v in x])
    assert np.array_equal(got8, bf)


@pytest.mark.parametrize("p,away", [(11, False), (11, True), (8, False)])
def test_tiered_reduces_to_plain_spamm(p, away):
    """tau_h <= tau (every kept product formed exactly) and p = 53 (no
    rounding) both give oracle_multiply's C bit for bit."""
    n, b, tau = 150, 16, 1e-3
    A = gen.exp_decay_nonsym(n, 0.8, seed=4)
    B = gen.exp_decay_nonsym(n, 0.85, seed=5)
    ref = O.multiply(A, B, b, tau)
    C, m, exact, rounded = O.multiply_tiered(A, B, b, tau, tau, p, away)
    assert np.array_equal(C, ref.C) and m == len(ref.triples) == exact and rounded == 0
    C, m, exact, rounded = O.multiply_tiered(A, B, b, tau, 1e9, 53, away)
    assert np.array_equal(C, ref.C) and rounded == m


def test_tiered_all_rounded_is_the_product_of_rounded_operands():
    """tau = 0 and tau_h above every norm product: every non-NULL leaf
    product is formed from operands rounded to 11 bits, so C is numpy's
    FP64 product of the float16-rounded matrices (within FP64 summation
    order)."""
    n, b = 200, 16
    A = gen.uniform_dense(n, seed=6, symmetric=False)
    B = gen.uniform_dense(n, seed=7, symmetric=False)
    # float16's subnormals keep fewer than 11 bits: stay in its normal range
    A[np.abs(A) < 2.0 ** -14] = 0.0
    B[np.abs(B) < 2.0 ** -14] = 0.0
    C, m, exact, rounded = O.multiply_tiered(A, B, b, 0.0, 1e30, 11)
    nl = -(-n // b)
    assert exact == 0 and rounded == m == nl ** 3
    ref = A.astype(np.float16).astype(np.float64) @ B.astype(np.float16).astype(np.float64)
    assert np.abs(C - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(C - A.astype(np.float64) @ B.astype(np.float64)).max() > 1e-5


@pytest.mark.parametrize("p,tau,shift", [(11, 1e-4, 10), (8, 1e-3, 7), (11, 1e-6, 14)])
def test_tiered_error_bound_and_counts(p, tau, shift):
    """||AB - C||_F <= sum over culled products of ||A_IK|| ||B_KJ|| plus
    (2u + u^2) times the same sum over the rounded ones (u = 2^-p); the
    exact and rounded counts are the kept products on either side of
    tau_h, recounted from numpy leaf norms."""
    n, b = 256, 16
    A = gen.exp_decay_nonsym(n, 0.85, seed=8)
    B = gen.exp_decay_nonsym(n, 0.8, seed=9)
    tau_h = tau * 2.0 ** shift
    C, m, exact, rounded = O.multiply_tiered(A, B, b, tau, tau_h, p)
    la, lb = _leaf_norm2(A, b), _leaf_norm2(B, b)
    P = la[:, :, None] * lb[None, :, :]
    pos = P > 0
    kept = pos & (P >= tau * tau)
    hi = kept & (P >= tau_h * tau_h)
    assert m == int(kept.sum()) and exact == int(hi.sum()) and rounded == m - exact
    assert 0 < exact < m
    u = 2.0 ** -p
    culled = np.sqrt(P[pos & ~kept]).sum()
    low = np.sqrt(P[kept & ~hi]).sum()
    err = np.linalg.norm(A.astype(np.float64) @ B.astype(np.float64) - C)
    assert err <= (culled + (2 * u + u * u) * low) * (1 + 1e-12)
    # the rounded tier alone, against plain SpAMM at the same tau: nonzero
    # and within (2u + u^2) times the rounded products' norm sum
    plain = O.multiply(A, B, b, tau).C
    diff = np.linalg.norm(C - plain)
    assert 0 < diff <= (2 * u + u * u) * low * (1 + 1e-12)


def test_sliced_tiered_with_one_slice_per_leaf_is_the_tiered_product():
    """The sub-leaf cull with one slice per leaf is plain SpAMM (R14), so
    with the precision tier it equals oracle_multiply_tiered bit for bit."""
    n, b, tau = 300, 32, 1e-4
    A = gen.exp_decay_nonsym(n, 0.85, seed=14)
    B = gen.exp_decay(n, 0.9, seed=15)
    tau_h = tau * 2.0 ** 10
    Ct, m, exact, rounded = O.multiply_tiered(A, B, b, tau, tau_h, 11)
    Cs, ms, kept, tested = O.multiply_sliced(A, B, b, b, tau, tau_h=tau_h, p=11)
    assert exact > 0 and rounded > 0
    assert np.array_equal(Cs, Ct) and ms == m and kept == tested == m


def test_tiered_blocks_match_the_tiered_product():
    """The sampled-block oracle with the precision tier equals the full
    tiered product block for block (same ascending-K order, same rounding)."""
    n, b, tau = 230, 16, 1e-4
    A = gen.exp_decay_nonsym(n, 0.85, seed=16)
    tau_h = tau * 2.0 ** 10
    for p, away in ((11, False), (11, True), (8, False)):
        C, _, exact, rounded = O.multiply_tiered(A, A, b, tau, tau_h, p, away)
        assert exact > 0 and rounded > 0
        ij = [(0, 0), (3, 7), (14, 14), (14, 0), (5, 9), (9, 5)]
        acc, _ = O.blocks(A, A, b, tau, ij, tau_h=tau_h, p=p, ties_away=away)
        for q, (I, J) in enumerate(ij):
            blk = C[I * b:min(n, (I + 1) * b), J * b:min(n, (J + 1) * b)]
            assert np.array_equal(acc[q][:blk.shape[0], :blk.shape[1]], blk)


# ------------------------------------- leaf-tier test == tier-by-tier (R17)
def _keep_grid(na, nb, tau):
    """The SpAMM predicate (R1-R3) on every (I, K, J) of two norm tiers."""
    a = na[:, :, None]
    b = nb[None, :, :]
    return (a > 0.0) & (b > 0.0) & (a * b >= tau * tau)


@pytest.mark.parametrize("n,b,tau,kind", [(300, 16, 1e-4, "exp"), (257, 8, 1e-3, "alg"),
                                          (128, 4, 0.0, "dense"), (200, 16, 3e-2, "exp"),
                                          (96, 2, 1e-2, "alg")])
def test_leaf_tier_test_gives_the_tier_by_tier_cull_and_its_counts(n, b, tau, kind):
    """R17: a leaf triple survives the level-by-level cull iff its own leaf
    norms pass (every ancestor's norm product is at least the leaf's), and
    tier t's tested triples are those whose parent passes, its kept ones
    those that pass themselves.  Both readings, evaluated directly on the
    oracle's pyramids, give the oracle's recursive triple set and per-tier
    counts exactly."""
    if kind == "exp":
        A, B = gen.exp_decay(n, 0.85, seed=1), gen.exp_decay_nonsym(n, 0.9, seed=2)
    elif kind == "alg":
        A, B = gen.algebraic_decay(n, seed=3), gen.algebraic_decay(n, seed=4)
    else:
        A, B = gen.uniform_dense(n, seed=5, symmetric=False), gen.uniform_dense(n, seed=6)
    ref = O.multiply(A, B, b, tau)
    pa, pb = O.pyramid(A, b), O.pyramid(B, b)
    d = O.depth(n, b)
    leaf = _keep_grid(O.tier(pa, d), O.tier(pb, d), tau)
    got = set(map(tuple, np.argwhere(leaf).tolist()))
    assert got == set(map(tuple, ref.triples.tolist()))
    cand, kept = [], []
    for t in range(d + 1):
        own = _keep_grid(O.tier(pa, t), O.tier(pb, t), tau)
        if t == 0:
            tested = np.ones_like(own)
        else:
            par = _keep_grid(O.tier(pa, t - 1), O.tier(pb, t - 1), tau)
            tested = par.repeat(2, 0).repeat(2, 1).repeat(2, 2)
        cand.append(int(tested.sum()))
        kept.append(int((tested & own).sum()))
        # kept iff passing itself: a passing triple's parent always passes
        assert int(own.sum()) == kept[-1]
    assert cand == ref.cand.tolist()
    assert kept == ref.kept.tolist()
