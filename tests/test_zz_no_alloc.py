"""tvolap_process_signal_static: the offline path for callers that must not
allocate device memory while running (a real-time audio callback, a process
under a fixed device-memory budget). It keeps its scratch in a fixed device
array. These tests call it through the C ABI and check it against the FP64
oracle (and against tvolap_process_signal) on two calls in a row, that the
second call leaves the device's free memory unchanged, that a request of
exactly the array's size works and one block more is refused, and that a
call with another device current than the plan's is refused.

Tolerance: relative L2 error <= 1e-5 and max-abs error <= 1e-4 x the oracle's
peak, the tolerance of the other GPU parity tests.
"""
import ctypes

import numpy as np
import pytest

import oracle
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STATIC_BYTES = 32 << 20          # TVOLAP_STATIC_SCRATCH_BYTES


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


def _static(lib, plan, wl, x, sa, sb, sal, y):
    return lib.tvolap_process_signal_static(plan.h, _p(x), wl.N, wl.N, _p(sa), _p(sb), _p(sal),
                                            sa.shape[1], _p(y), wl.out_len, wl.out_len)


def _inputs(wl, dev):
    return (torch.from_numpy(wl.x).to(dev), torch.from_numpy(wl.sched_a).to(dev),
            torch.from_numpy(wl.sched_b).to(dev), torch.from_numpy(wl.sched_alpha).to(dev))


def _oracle(wl):
    return oracle.tvolap_direct(wl.x, wl.irs, wl.L, wl.sched_a, wl.sched_b, wl.sched_alpha,
                                out_len=wl.out_len, out_to_in=list(wl.out_to_in))


def test_static_scratch_entry_point_matches_oracle():
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
        x, sa, sb, sal = _inputs(wl, dev)
        lib_y = plan.process_signal(x, sa, sb, sal, out_len=wl.out_len).cpu().numpy()
        y = torch.full((3, wl.out_len), float("nan"), device=dev)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info(dev)[0]
        st = _static(lib, plan, wl, x, sa, sb, sal, y)
        assert st == 0, _lib.STATUS.get(st, st)
        plan.check()
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info(dev)[0]
        if i > 0:
            # the array was set up by the first call: this call took no device memory
            assert free_after == free_before
        got = y.cpu().numpy()
        _close(got, _oracle(wl))
        _close(got, lib_y)
        plan.close()


def test_static_scratch_at_capacity_and_one_block_beyond():
    """One input and one output at L = 128: 8 * P * n_blocks * 2 bytes equals
    the array's size at n_blocks = 8192 (out_len up to 8191 * 128); that call
    runs and matches the oracle, and one sample more (8193 blocks) is refused
    with TVOLAP_ERR_CAPACITY and leaves the output untouched."""
    dev = _dev()
    from paper_2310_00319_gb300 import Plan, _lib
    lib = _lib.load()
    L, P = 128, 256
    nb = STATIC_BYTES // (8 * P * 2)
    assert nb == 8192
    out_len = (nb - 1) * L                             # the largest length with nb blocks
    wl = W.random_case(503, L=L, ir_len=400, N=out_len, n_in=1, n_out=1, n_slots=3,
                       out_len=out_len)
    assert wl.sched_a.shape[1] == nb
    plan = Plan(L, wl.M, n_in=1, n_out=1, n_slots=3, device=dev)
    plan.load_bank(0, torch.from_numpy(wl.irs).to(dev))
    x, sa, sb, sal = _inputs(wl, dev)
    y = torch.full((1, out_len), float("nan"), device=dev)
    st = _static(lib, plan, wl, x, sa, sb, sal, y)
    assert st == 0, _lib.STATUS.get(st, st)
    plan.check()
    _close(y.cpu().numpy(), _oracle(wl))
    # one block more
    big = W.random_case(504, L=L, ir_len=400, N=out_len + 1, n_in=1, n_out=1, n_slots=3,
                        out_len=out_len + 1)
    assert big.sched_a.shape[1] == nb + 1
    x, sa, sb, sal = _inputs(big, dev)
    y2 = torch.full((1, out_len + 1), 7.0, device=dev)
    st = _static(lib, plan, big, x, sa, sb, sal, y2)
    assert st == -5                                     # TVOLAP_ERR_CAPACITY
    torch.cuda.synchronize()
    assert torch.all(y2 == 7.0)
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


def test_static_scratch_refuses_another_current_device():
    """The plan's device (its stream's) must be current: with another device
    current the call is refused (TVOLAP_ERR_ARG). Needs two GPUs."""
    dev = _dev()
    if torch.cuda.device_count() < 2:
        pytest.skip("needs a second GPU")
    from paper_2310_00319_gb300 import Plan, _lib
    lib = _lib.load()
    wl = W.random_case(505, L=64, ir_len=300, N=2000, n_in=1, n_out=1, n_slots=2)
    plan = Plan(64, wl.M, n_in=1, n_out=1, n_slots=2, device=dev)
    plan.load_bank(0, torch.from_numpy(wl.irs).to(dev))
    x, sa, sb, sal = _inputs(wl, dev)
    y = torch.zeros((1, wl.out_len), device=dev)
    with torch.cuda.device(1):
        st = _static(lib, plan, wl, x, sa, sb, sal, y)
    assert st == -1                                     # TVOLAP_ERR_ARG
    plan.close()
