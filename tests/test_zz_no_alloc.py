"""The allocation-free coarsest solve (mgmlmc_coarse_inverse_noalloc).

Some callers cannot allocate device memory while they run (a host framework that
owns a fixed memory budget, a real-time loop that cannot take cudaMalloc's
synchronisation).  The entry point gives them the
mixed-precision coarsest solve with its work space in a static device array; the
caller passes device input and output.  Checked against mgmlmc_apply(OP_DINV_C),
which runs the same tensor-core kernel with context work space, on two calls in
a row (the second one reuses the static array left over from the first).

This file is collected last on purpose, and it sets up everything it needs, so it
passes both alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

# Same computation on the same FP32 input: equal up to FP32 rounding of the
# accumulation order (the context path may split the sum over n_L) and of the
# returned values (the host path converts to FP64 and back).
TOL = 1e-6


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2211_15383_gb300 as pkg
    return torch, pkg


def _ctx(pkg, precision):
    w = inputs.workload("schwinger-16x16")
    ctx = pkg.Context(mg_precision=precision)
    ctx.set_gauge(w.gauge())
    ctx.set_mass(w.m0)
    ctx.set_hierarchy(w.agg, w.nvec, w.start_vectors(), setup_iters=0)
    return ctx


@pytest.mark.parametrize("precision,nrhs", [(32, 64), (32, 256), (16, 64)])
def test_noalloc_matches_existing_entry_point(env, precision, nrhs):
    torch, pkg = env
    with _ctx(pkg, precision) as ctx:
        n = ctx.level_info(2)[3]
        rng = np.random.default_rng(nrhs)
        x = (rng.standard_normal((nrhs, n)) + 1j * rng.standard_normal((nrhs, n))).astype(np.complex64)
        ref = ctx.apply(pkg.OP_DINV_C, 2, x.astype(np.complex128), n)
        # caller-owned device buffers, layout [n_L][nrhs] complex64
        xd = torch.from_numpy(np.ascontiguousarray(x.T)).cuda()
        stream = torch.cuda.current_stream()
        for _call in range(2):
            yd = torch.full((n, nrhs), float("nan"), dtype=torch.complex64, device="cuda")
            torch.cuda.synchronize()
            ctx.coarse_inverse_noalloc(nrhs, xd.data_ptr(), yd.data_ptr(), stream.cuda_stream)
            y = yd.cpu().numpy().T.astype(np.complex128)
            assert np.all(np.isfinite(y))
            assert np.abs(y - ref).max() <= TOL * np.abs(ref).max()


def test_noalloc_limits(env):
    torch, pkg = env
    with _ctx(pkg, 32) as ctx:
        n = ctx.level_info(2)[3]
        buf = torch.zeros((n, 4096), dtype=torch.complex64, device="cuda")
        out = torch.zeros_like(buf)
        with pytest.raises(pkg.MgmlmcError) as e:          # not a multiple of 32
            ctx.coarse_inverse_noalloc(33, buf.data_ptr(), out.data_ptr())
        assert e.value.code == -1
        too_many = 32 * ((2 ** 20 // n) // 32 + 1)           # n_L * nrhs above 2^20
        with pytest.raises(pkg.MgmlmcError) as e:
            ctx.coarse_inverse_noalloc(too_many, buf.data_ptr(), out.data_ptr())
        assert e.value.code == -1
        # y off its 16-byte alignment (one complex64 in): refused on the host, no kernel runs
        with pytest.raises(pkg.MgmlmcError) as e:
            ctx.coarse_inverse_noalloc(32, buf.data_ptr(), out.data_ptr() + 8)
        assert e.value.code == -1
    with _ctx(pkg, 64) as ctx:                              # FP64 mode keeps no BF16 inverse
        n = ctx.level_info(2)[3]
        buf = torch.zeros((n, 32), dtype=torch.complex64, device="cuda")
        out = torch.zeros_like(buf)
        with pytest.raises(pkg.MgmlmcError) as e:
            ctx.coarse_inverse_noalloc(32, buf.data_ptr(), out.data_ptr())
        assert e.value.code == -8
