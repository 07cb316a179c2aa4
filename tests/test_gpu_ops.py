"""GPU operator parity against the oracle: D_l, P^H, P, Gamma5, the coarsest
inverse and the Z2 noise, on seeded inputs of several sizes (ragged rhs counts)."""
import numpy as np
import pytest

from oracle import hierarchy as ohier
from oracle import noise as onoise
from oracle import wilson as owilson

from gpu_common import make_ctx, rand_complex, require_gpu, small_problem

pytestmark = pytest.mark.gpu

CASES = [
    # (Lx, Lt, agg, nvec)
    (8, 8, ((2, 2), (2, 2)), (2, 2)),
    (16, 16, ((4, 4),), (4,)),
    (12, 8, ((2, 4), (3, 1)), (2, 3)),
    (16, 8, ((4, 4),), (8,)),            # d = 16 on the coarse level
]


@pytest.fixture(scope="module")
def pkg():
    return require_gpu()


@pytest.mark.parametrize("Lx,Lt,agg,nvec", CASES)
@pytest.mark.parametrize("nrhs", [1, 3, 37, 70])
def test_operators_match_oracle(pkg, Lx, Lt, agg, nvec, nrhs):
    m0 = 0.05
    theta, sv = small_problem(Lx, Lt, agg=agg, nvec=nvec)
    H = ohier.build_hierarchy(theta, m0, agg, nvec, sv, 0)
    rng = np.random.default_rng(Lx * 100 + nrhs)
    with make_ctx(pkg, theta, m0, agg, nvec, sv, 0) as ctx:
        for lev in range(1, H.nlevels + 1):
            n = H.D[lev - 1].shape[0]
            x = rand_complex(rng, (nrhs, n))
            y = ctx.apply(pkg.OP_D, lev, x, n)
            ref = (H.D[lev - 1] @ x.T).T
            assert np.abs(y - ref).max() < 1e-13 * np.abs(ref).max(), f"D_{lev}"
            g = ctx.apply(pkg.OP_G5, lev, x, n)
            assert np.array_equal(g, H.g5[lev - 1][None, :] * x)
            if lev < H.nlevels:
                P = H.P[lev - 1]
                nc = P.shape[1]
                yc = ctx.apply(pkg.OP_PH, lev, x, nc)
                refc = (P.conj().T @ x.T).T
                assert np.abs(yc - refc).max() < 1e-13 * np.abs(refc).max(), f"P^H_{lev}"
                xc = rand_complex(rng, (nrhs, nc))
                yf = ctx.apply(pkg.OP_P, lev, xc, n)
                reff = (P @ xc.T).T
                assert np.abs(yf - reff).max() < 1e-13 * np.abs(reff).max(), f"P_{lev}"
        # the coarsest level's stored inverse
        L = H.nlevels
        n = H.D[-1].shape[0]
        b = rand_complex(rng, (nrhs, n))
        z = ctx.apply(pkg.OP_DINV_C, L, b, n)
        ref = np.linalg.solve(H.D[-1].toarray(), b.T).T
        assert np.abs(z - ref).max() < 1e-10 * np.abs(ref).max()


def test_free_field_fine_operator(pkg):
    # theta = 0: the fine operator against the oracle at a non-square size
    Lx, Lt, m0 = 6, 10, 0.3
    theta = np.zeros((Lt, Lx, 2))
    _, sv = small_problem(Lx, Lt, agg=((3, 5),), nvec=(1,))
    with make_ctx(pkg, theta, m0, ((3, 5),), (1,), sv, 0) as ctx:
        D = owilson.wilson_dirac(theta, m0)
        x = rand_complex(np.random.default_rng(1), (5, D.shape[0]))
        y = ctx.apply(pkg.OP_D, 1, x, D.shape[0])
        assert np.abs(y - (D @ x.T).T).max() < 1e-13


@pytest.mark.parametrize("first,ns", [(0, 1), (5, 33), (1000, 70)])
def test_noise_bit_exact(pkg, first, ns):
    theta, sv = small_problem()
    with make_ctx(pkg, theta, 0.05, ((2, 2), (2, 2)), (2, 2), sv, 0) as ctx:
        for lev in (1, 2, 3):
            n = ctx.level_info(lev)[3]
            x = ctx.noise(lev, first, ns, 0xABCDEF0123)
            ref = onoise.z2_noise(0xABCDEF0123, lev, first, ns, n)
            assert np.array_equal(x, ref)


def test_rank_deficient_test_vectors_rejected(pkg):
    theta, sv = small_problem(agg=((2, 2),), nvec=(2,))
    sv = [np.stack([sv[0][0], 2.0 * sv[0][0]])]            # second vector parallel to the first
    with pkg.Context() as ctx:
        ctx.set_gauge(theta)
        ctx.set_mass(0.05)
        with pytest.raises(pkg.MgmlmcError) as e:
            ctx.set_hierarchy(((2, 2),), (2,), sv, setup_iters=0)
        assert e.value.code == -1


def test_state_errors(pkg):
    with pkg.Context() as ctx:
        with pytest.raises(pkg.MgmlmcError) as e:
            ctx.estimate_level(0, 0, 4, 1)
        assert e.value.code == -8
        with pytest.raises(pkg.MgmlmcError):
            ctx.set_gauge(np.zeros((3, 4, 2)))          # odd Lt
        bad = np.zeros((4, 4, 2))
        bad[0, 0, 0] = np.nan
        with pytest.raises(pkg.MgmlmcError) as e:
            ctx.set_gauge(bad)
        assert e.value.code == -7


@pytest.mark.parametrize("nrhs", [1, 3, 37, 64, 130, 256])
def test_tensor_core_coarsest_solve(pkg, nrhs):
    # mixed mode: the coarsest inverse is rounded to BF16 and applied with tcgen05 MMAs
    # (FP32 accumulation); compare with the exact solve at BF16 accuracy
    import inputs
    w = inputs.workload("schwinger-16x16")
    theta, sv = w.gauge(), w.start_vectors()
    H = ohier.build_hierarchy(theta, w.m0, w.agg, w.nvec, sv, 0)
    n = H.D[-1].shape[0]
    assert n % 128 == 0
    rng = np.random.default_rng(nrhs)
    b = rand_complex(rng, (nrhs, n))
    ref = np.linalg.solve(H.D[-1].toarray(), b.T).T
    with make_ctx(pkg, theta, w.m0, w.agg, w.nvec, sv, 0, mg_precision=32) as ctx:
        z = ctx.apply(pkg.OP_DINV_C, 2, b, n)
        z2 = ctx.apply(pkg.OP_DINV_C, 2, b, n)
    assert np.array_equal(z, z2)                                   # deterministic
    assert np.linalg.norm(z - ref) / np.linalg.norm(ref) < 2e-2
    # per rhs as well (no column is left unwritten or mixed up)
    err = np.linalg.norm(z - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() < 3e-2


def _round_bf16(a):
    """Round float32 values to BF16 (round to nearest, ties to even), as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (u & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)


def _round_c(z, bf16):
    """Complex values as the GPU sees them: FP32, then (bf16) BF16 per part."""
    z = np.asarray(z).astype(np.complex64)
    if not bf16:
        return z.astype(np.complex128)
    return _round_bf16(z.real) + 1j * _round_bf16(z.imag)


@pytest.mark.parametrize("prec", [64, 32, 16])
@pytest.mark.parametrize("nrhs", [1, 37, 130, 300, 600])
def test_smoother_operator(pkg, prec, nrhs):
    # y = D_2 M_2^{-1} x, M_2 = block diagonal (self blocks) of D_2, on a level with
    # d = 16 (4 x 4 sites): FP64 / FP32 block stencils, and (prec 16) the tcgen05
    # kernel on BF16 tiles of 128 rhs (1, 37 and 130 leave a ragged tile, 300 and
    # 600 a ragged third / fifth one), whose result must equal the same products
    # of the BF16-rounded operands up to FP32 accumulation
    import scipy.sparse as sp
    agg, nvec = ((4, 4), (2, 2)), (8, 8)
    theta, sv = small_problem(16, 16, agg=agg, nvec=nvec)
    H = ohier.build_hierarchy(theta, 0.05, agg, nvec, sv, 0)
    D2 = H.D[1].tocsr()
    n, d = D2.shape[0], 16
    blocks = [np.linalg.inv(D2[s * d:(s + 1) * d, s * d:(s + 1) * d].toarray()) for s in range(n // d)]
    Ahat = (D2 @ sp.block_diag([sp.csr_matrix(b) for b in blocks], format="csr")).tocsr()
    rng = np.random.default_rng(1000 + nrhs)
    x = rand_complex(rng, (nrhs, n))
    ref = (Ahat @ x.T).T
    with make_ctx(pkg, theta, 0.05, agg, nvec, sv, 0, mg_precision=prec) as ctx:
        ctx.profile(True, reset=True)
        y = ctx.apply(pkg.OP_SMOOTH, 2, x, n)
        y2 = ctx.apply(pkg.OP_SMOOTH, 2, x, n)
        classes = set(ctx.profile_report())
        ctx.profile(False)
        # the kernel class that ran: BF16 tensor cores exactly when prec 16
        assert ("D2.bf16" in classes) == (prec == 16), classes
        with pytest.raises(pkg.MgmlmcError):
            ctx.apply(pkg.OP_SMOOTH, 3, x[:, :64], 64)            # the coarsest level has no smoother
    assert np.array_equal(y, y2)
    scale = np.abs(ref).max()
    if prec == 64:
        assert np.abs(y - ref).max() < 1e-12 * scale
        return
    if prec == 32:
        assert np.abs(y - ref).max() < 2e-5 * scale
        return
    # BF16 operands: the embedding (signs, layouts, neighbours) is pinned by the
    # emulated products, the accuracy by the exact operator
    Ab = Ahat.copy()
    Ab.data = _round_c(Ab.data, True)
    emu = (Ab @ _round_c(x, True).T).T
    assert np.abs(y - emu).max() < 2e-5 * scale
    rel = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rel.max() < 1.5e-2
