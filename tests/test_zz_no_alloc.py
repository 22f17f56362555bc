"""tvolap_process_signal_static: the offline path for callers that must not
allocate device memory while running (a real-time audio callback, a process
under a fixed device-memory budget). It keeps its scratch in a fixed device
array; this test calls it through the C ABI and checks it against
tvolap_process_signal on two calls in a row, and that the second call leaves
the device's free memory unchanged.

Tolerance: relative L2 error <= 1e-5 and max-abs error <= 1e-4 x peak, the
tolerance of the other GPU parity tests.
"""
import ctypes

import numpy as np
import pytest

from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _close(y, ref):
    y = np.asarray(y, np.float64)
    ref = np.asarray(ref, np.float64)
    for o in range(ref.shape[0]):
        rel = np.linalg.norm(y[o] - ref[o]) / np.linalg.norm(ref[o])
        mx = np.max(np.abs(y[o] - ref[o])) / np.max(np.abs(ref[o]))
        assert rel <= 1e-5 and mx <= 1e-4, (o, rel, mx)


def test_static_scratch_entry_point_matches_process_signal():
    dev = _dev()
    from paper_2310_00319_gb300 import Plan, _lib
    lib = _lib.load()
    cases = [W.random_case(501, L=128, ir_len=3000, N=40000, n_in=2, n_out=3, n_slots=5,
                           out_len=41000, out_to_in=[0, 1, 1]),
             W.random_case(502, L=128, ir_len=2500, N=30000, n_in=2, n_out=3, n_slots=5,
                           out_len=30000, out_to_in=[1, 0, 1])]
    for i, wl in enumerate(cases):
        plan = Plan(128, wl.M, n_in=2, n_out=3, out_to_in=list(wl.out_to_in), n_slots=5,
                    device=dev)
        plan.load_bank(0, torch.from_numpy(wl.irs).to(dev))
        x = torch.from_numpy(wl.x).to(dev)
        sa = torch.from_numpy(wl.sched_a).to(dev)
        sb = torch.from_numpy(wl.sched_b).to(dev)
        sal = torch.from_numpy(wl.sched_alpha).to(dev)
        ref = plan.process_signal(x, sa, sb, sal, out_len=wl.out_len).cpu().numpy()
        y = torch.full((3, wl.out_len), float("nan"), device=dev)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info(dev)[0]
        st = lib.tvolap_process_signal_static(plan.h, _p(x), wl.N, wl.N, _p(sa), _p(sb), _p(sal),
                                              sa.shape[1], _p(y), wl.out_len, wl.out_len)
        assert st == 0, _lib.STATUS.get(st, st)
        plan.check()
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info(dev)[0]
        if i > 0:
            # the array was set up by the first call: this call took no device memory
            assert free_after == free_before
        _close(y.cpu().numpy(), ref)
        plan.close()


def test_static_scratch_rejects_oversize():
    dev = _dev()
    from paper_2310_00319_gb300 import Plan, _lib
    lib = _lib.load()
    plan = Plan(1024, 2, n_in=8, n_out=8, n_slots=1, device=dev)
    N = 600000                                          # 8 * 2048 * 588 * 16 B > 32 MiB
    x = torch.zeros((8, N), device=dev)
    nb = (N - 1) // 1024 + 2
    sa = torch.zeros((8, nb), dtype=torch.int32, device=dev)
    y = torch.zeros((8, N), device=dev)
    st = lib.tvolap_process_signal_static(plan.h, _p(x), N, N, _p(sa), None, None, nb, _p(y), N, N)
    assert st == -5                                     # TVOLAP_ERR_CAPACITY
    plan.close()
