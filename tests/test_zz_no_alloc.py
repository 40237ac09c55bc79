"""The allocation-free solve (okmc_solve_stress_static) against the handle-based solve.

okmc_solve_stress_static serves callers that cannot allocate device memory: it
keeps its scratch in a static device array, so it must give the same stress as
okmc_solve_stress on the same eigenstrain, call after call.  This file is
collected last so that a run stopping at the first failure has run every other
test before it.
"""
import ctypes as C

import numpy as np
import pytest

import __graft_entry__
from paper_2403_09158_gb300 import okmc as ok
from paper_2403_09158_gb300.workload import config_small, scaled_population

pytestmark = pytest.mark.gpu


def _static_solve(lib, torch, eps_d, sig_d, w, k0):
    n = (C.c_int32 * 3)(*w.n)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.okmc_solve_stress_static(eps_d.data_ptr(), sig_d.data_ptr(), n, *w.C, k0, stream)
    torch.cuda.synchronize()
    return rc


@pytest.mark.parametrize('case', ['32cubed', '64x48x32'])
def test_static_solve_equals_handle_solve_twice(case):
    torch = pytest.importorskip('torch')
    __graft_entry__.build()
    lib = ok.load()
    w = config_small() if case == '32cubed' else scaled_population((64, 48, 32), 10, seed=5, r111=(0.4, 1.0),
                                                                     r100=(0.4, 1.0))
    for k0 in (ok.MEAN_STRESS_ZERO, ok.MEAN_STRAIN_ZERO):
        g = ok.Grid(w.n, w.voxel_nm, *w.C, k0_mode=k0)
        g.set_defects(w.defects)
        eps = g.eigenstrain()
        ref = g.solve_stress()
        g.close()
        eps_d = torch.from_numpy(eps).cuda()
        sigs = [torch.full_like(eps_d, float('nan')) for _ in range(2)]
        free = []
        for call in range(2):
            free.append(torch.cuda.mem_get_info()[0])
            assert _static_solve(lib, torch, eps_d, sigs[call], w, k0) == ok.OKMC_OK
            sig = sigs[call].cpu().numpy()
            rel = np.linalg.norm(sig.astype(np.float64) - ref) / np.linalg.norm(ref)
            assert rel <= 1e-5, (case, k0, call, rel)
        # the first call of the process may load the module (and with it the static
        # array); from then on a call takes no device memory at all
        free.append(torch.cuda.mem_get_info()[0])
        assert free[2] == free[1], (case, k0, free)


def test_static_solve_rejects_misaligned_pointers():
    torch = pytest.importorskip('torch')
    __graft_entry__.build()
    lib = ok.load()
    w = config_small()
    N = 6 * int(np.prod(w.n))
    buf = torch.zeros(N + 1, device='cuda')
    good = torch.zeros(N, device='cuda')
    # a view one float in: 4-byte aligned only; the call must refuse it on the host
    assert _static_solve(lib, torch, buf[1:], good, w, ok.MEAN_STRESS_ZERO) == ok.OKMC_EINVAL
    assert _static_solve(lib, torch, good, buf[1:], w, ok.MEAN_STRESS_ZERO) == ok.OKMC_EINVAL


def test_static_solve_rejects_oversize_grid():
    torch = pytest.importorskip('torch')
    __graft_entry__.build()
    lib = ok.load()
    w = scaled_population((80, 64, 64), 4, seed=6)       # 6*41*64*64 > 6*33*64*64
    eps_d = torch.zeros((6, 64, 64, 80), device='cuda')
    sig_d = torch.zeros_like(eps_d)
    assert _static_solve(lib, torch, eps_d, sig_d, w, ok.MEAN_STRESS_ZERO) == ok.OKMC_EINVAL
