"""Host-side checks of the request server (no GPU work): its admission policy, the
layout of every C struct the binding mirrors, and the footprint model's argument
checks and monotonicity."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2211_15383_gb300", "csrc")


def _cxx():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    return cxx


def test_admission_policy(tmp_path):
    exe = str(tmp_path / "admission_check")
    subprocess.run([_cxx(), "-std=c++17", "-O1", "-Wall", "-I", CSRC, os.path.join(ROOT, "tests", "admission_check.cpp"),
                    "-o", exe], check=True)
    res = subprocess.run([exe], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout + res.stderr


def _structs():
    from paper_2211_15383_gb300 import _lib
    return {"mgmlmc_options": _lib.Options, "mgmlmc_level_stats": _lib.LevelStats,
            "mgmlmc_trace_result": _lib.TraceResult, "mgmlmc_server_options": _lib.ServerOptions,
            "mgmlmc_request": _lib.Request, "mgmlmc_request_result": _lib.RequestResult,
            "mgmlmc_server_stats": _lib.ServerStats, "mgmlmc_tune_result": _lib.TuneResult,
            "mgmlmc_tune_trial": _lib.TuneTrial}


def test_struct_layout_matches_header(tmp_path):
    # offsets and sizes of the C structs (compiled against include/mgmlmc.h) against
    # the ctypes mirrors of the binding
    structs = _structs()
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mgmlmc.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "layout")
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    seen = 0
    for line in out:
        if not line:
            continue
        cname, field, val = line.split()
        py = structs[cname]
        want = ctypes.sizeof(py) if field == "sizeof" else getattr(py, field).offset
        assert int(val) == want, f"{cname}.{field}: C {val}, ctypes {want}"
        seen += 1
    assert seen == sum(len(p._fields_) + 1 for p in structs.values())


def _request(pkg, L, agg, nvec, k=0, **kw):
    th = np.zeros((L, L, 2))
    sv, lx, d = [], L, 2
    for (a, _), nv in zip(agg, nvec):
        sv.append(np.zeros((nv, lx * lx * d), np.complex128))
        lx //= a
        d = 2 * nv
    return pkg.make_request(th, -0.1, agg, nvec, sv, 1e-3, 1, k=k, **kw)


@pytest.fixture(scope="module")
def pkg():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2211_15383_gb300 import build
    build.build()
    import paper_2211_15383_gb300 as p
    p.load()
    return p


def test_request_footprint_checks_and_grows(pkg):
    base = pkg.request_footprint(_request(pkg, 64, [(4, 4), (2, 2)], [8, 8], k=32, mg_precision=16))
    assert base > 0
    # more right-hand sides per block, a larger lattice, FP64 V-cycle, more triplets: more bytes
    assert pkg.request_footprint(_request(pkg, 64, [(4, 4), (2, 2)], [8, 8], k=32, mg_precision=16,
                                          max_block_rhs=512)) > base
    assert pkg.request_footprint(_request(pkg, 128, [(4, 4), (2, 2)], [8, 8], k=32, mg_precision=16)) > base
    assert pkg.request_footprint(_request(pkg, 64, [(4, 4), (2, 2)], [8, 8], k=32, mg_precision=64)) > base
    assert pkg.request_footprint(_request(pkg, 64, [(4, 4), (2, 2)], [8, 8], k=128, mg_precision=16)) > base
    # the Krylov bases of the finest level alone are a lower bound: (2m + 1) n_1 N * 8 B
    n1, N, m = 64 * 64 * 2, 256, 24
    assert base > (2 * m + 1) * n1 * N * 8
    # malformed hierarchies are refused as set_hierarchy refuses them
    with pytest.raises(pkg.MgmlmcError) as e:
        pkg.request_footprint(_request(pkg, 64, [(5, 4)], [4]))             # 5 does not divide 64
    assert e.value.code == -1
    with pytest.raises(pkg.MgmlmcError) as e:
        pkg.request_footprint(_request(pkg, 16, [(2, 2)], [8]))             # 8 > 2*2*2/2 rows
    assert e.value.code == -1
    with pytest.raises(pkg.MgmlmcError) as e:
        pkg.request_footprint(_request(pkg, 256, [(4, 4)], [8]))            # coarsest 64^2 * 16 > 16384
    assert e.value.code == -6
    with pytest.raises(pkg.MgmlmcError) as e:
        pkg.request_footprint(_request(pkg, 64, [(4, 4)], [8], mg_precision=8))   # options as mgmlmc_create
    assert e.value.code == -1 and "mg_precision" in str(e.value)


def test_footprint_of_deep_solver_hierarchies(pkg):
    # the 1024^2 workload: a 3-term sum over 6 levels (three solver-only levels),
    # 512 triplets of level 3; the model must admit one block of 128 rhs with
    # restart 16 on a 288 GB GPU and refuse 1024 rhs with restart 24, which is how
    # the autotuner's candidates are bounded
    agg, nvec = [(4, 4), (2, 2), (2, 2), (2, 2), (2, 2)], [8] * 5
    small = pkg.request_footprint(_request(pkg, 1024, agg, nvec, k=512, mg_precision=16, sum_levels=3,
                                           max_block_rhs=128, fgmres_restart=16))
    big = pkg.request_footprint(_request(pkg, 1024, agg, nvec, k=512, mg_precision=16, sum_levels=3,
                                         max_block_rhs=1024, fgmres_restart=24))
    assert small < 250e9 < big
    # the deflated level is level 3 (262144 unknowns): more triplets cost more there
    more = pkg.request_footprint(_request(pkg, 1024, agg, nvec, k=1024, mg_precision=16, sum_levels=3,
                                          max_block_rhs=128, fgmres_restart=16))
    assert more - small > 2 * 262144 * 512 * 16
    # a K-cycle keeps extra Krylov bases on the coarse levels
    kc = pkg.request_footprint(_request(pkg, 1024, agg, nvec, k=512, mg_precision=16, sum_levels=3,
                                        max_block_rhs=128, fgmres_restart=16, kcycle_iters=2))
    assert kc > small
    with pytest.raises(pkg.MgmlmcError) as e:
        pkg.request_footprint(_request(pkg, 64, [(4, 4), (2, 2)], [8, 8], sum_levels=4))   # > nlevels
    assert e.value.code == -1


def test_server_calls_without_a_device(pkg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    lib = pkg.load()
    h = ctypes.c_void_p()
    assert lib.mgmlmc_server_create(ctypes.byref(h), None) == -5          # no device
    assert not h.value
    assert b"no CUDA device" in lib.mgmlmc_server_last_error(None)
    assert lib.mgmlmc_submit(None, None, None) == -1
    assert lib.mgmlmc_cancel(None, 1) == -1
    lib.mgmlmc_server_destroy(None)
