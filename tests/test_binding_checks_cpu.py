"""The Python binding checks every tensor's dtype, device and extents before
it hands a pointer to the C ABI (the kernels index those extents, so a smaller
tensor would be read or written out of bounds). Run on CPU with the ABI call
replaced by a recorder: a wrong shape must raise before any call, the right
shape must reach it."""
import types

import numpy as np
import pytest
import torch

from paper_2310_00319_gb300.batch import BatchedTvolap
from paper_2310_00319_gb300.nonuniform import NonUniform
from paper_2310_00319_gb300.server import Server
from paper_2310_00319_gb300.tvolap import Plan, n_blocks_for

L, M, N_IN, N_OUT, N_MIX = 16, 3, 2, 3, 2
P = 2 * L
C64, F32, I32, I64 = torch.complex64, torch.float32, torch.int32, torch.int64


def _recorder(obj):
    obj.calls = []
    obj._call = lambda name, *a: obj.calls.append(name) or 0
    return obj


@pytest.fixture
def plan():
    p = object.__new__(Plan)
    p.L, p.M, p.P, p.n_in, p.n_out, p.n_mix = L, M, P, N_IN, N_OUT, N_MIX
    p.device = torch.device("cpu")
    return _recorder(p)


def z(shape, dt=F32):
    return torch.zeros(shape, dtype=dt)


def _reaches(p, name, fn):
    fn()
    assert p.calls and p.calls[-1] == name


def _refused(p, fn, exc=ValueError):
    n = len(p.calls)
    with pytest.raises(exc):
        fn()
    assert len(p.calls) == n, "reached the C ABI"


def test_process_block_extents(plan):
    x = z((N_IN, L))
    _reaches(plan, "tvolap_process_block", lambda: plan.process_block(x, z((N_OUT, L))))
    _reaches(plan, "tvolap_process_block",
             lambda: plan.process_block(x, None, z(N_OUT, I32), z(N_OUT, I32), z(N_OUT)))
    for out in (z((N_OUT - 1, L)), z((N_OUT, L // 2)), z((N_OUT, L), C64)):
        _refused(plan, lambda: plan.process_block(x, out), (ValueError, TypeError))
    _refused(plan, lambda: plan.process_block(x, None, z(N_OUT - 1, I32)))
    _refused(plan, lambda: plan.process_block(z((N_IN, L + 1))))


def test_mixdown_extents(plan):
    x = z((N_IN, L))
    _reaches(plan, "tvolap_process_block_mix", lambda: plan.process_block_mix(x, z((N_MIX, L))))
    _refused(plan, lambda: plan.process_block_mix(x, z((N_OUT, L))))
    Y = z((N_OUT, 5, P), C64)
    _reaches(plan, "tvolap_mix", lambda: plan.mix(Y))
    _reaches(plan, "tvolap_mix", lambda: plan.mix(Y, z((N_MIX, 5, P), C64)))
    for bad in (z((N_OUT - 1, 5, P), C64), z((N_OUT, 5, P // 2), C64)):
        _refused(plan, lambda: plan.mix(bad))
    _refused(plan, lambda: plan.mix(Y, z((N_MIX, 4, P), C64)))


def test_stage_entry_point_extents(plan):
    nb = 6
    sched = z((N_OUT, nb), I32)
    _reaches(plan, "tvolap_forward_spectra", lambda: plan.forward_spectra(z((N_IN, 80)), nb))
    _refused(plan, lambda: plan.forward_spectra(z((N_IN + 1, 80)), nb))
    _reaches(plan, "tvolap_mac", lambda: plan.mac(z((N_IN, nb, P), C64), sched))
    for bad in (z((N_IN + 1, nb, P), C64), z((N_IN, nb, P - 2), C64)):
        _refused(plan, lambda: plan.mac(bad, sched))
    _refused(plan, lambda: plan.mac(z((N_IN, nb + 1, P), C64), sched))     # schedule too short
    out_len = (nb - 2) * L + 1
    assert n_blocks_for(out_len, L) == nb
    _reaches(plan, "tvolap_inverse_ola", lambda: plan.inverse_ola(z((N_OUT, nb, P), C64), out_len))
    _refused(plan, lambda: plan.inverse_ola(z((N_IN, nb, P), C64), out_len))


def test_ragged_extents(plan):
    nb = n_blocks_for(100, L)
    args = dict(x=z((N_IN, 100)), n=z(N_IN, I64), out_len=z(N_OUT, I64), parts=z(N_OUT, I32),
                max_out_len=100, sched_a=z((N_OUT, nb), I32))
    _reaches(plan, "tvolap_process_ragged", lambda: plan.process_ragged(**args))
    for k, bad in (("n", z(N_IN + 1, I64)), ("out_len", z(N_OUT - 1, I64)),
                   ("parts", z(N_OUT + 1, I32)), ("x", z((N_IN + 1, 100))),
                   ("out", z((N_OUT - 1, 100)))):
        _refused(plan, lambda: plan.process_ragged(**{**args, k: bad}))


def test_differentiable_extents(plan):
    nb, pb = 6, 6
    x, g = z((N_IN, 90)), z((N_OUT, 90))
    Pspec = z((N_OUT, pb, M, P), C64)
    X = z((N_IN, nb, P), C64)
    G = z((N_OUT, nb, P), C64)
    _reaches(plan, "tvolap_block_spectra", lambda: plan.block_spectra(x, 0, nb))
    _refused(plan, lambda: plan.block_spectra(z((N_IN + 1, 90)), 0, nb))
    _reaches(plan, "tvolap_mac_params", lambda: plan.mac_params(X, 0, Pspec, 0, nb))
    _refused(plan, lambda: plan.mac_params(X, 0, z((N_OUT, pb, M - 1, P), C64), 0, nb))
    _refused(plan, lambda: plan.mac_params(X, 0, Pspec, 0, nb, out=z((N_OUT, nb, P // 2), C64)))
    _reaches(plan, "tvolap_adjoint_output", lambda: plan.adjoint_output(g, 0, nb))
    _refused(plan, lambda: plan.adjoint_output(x, 0, nb))
    dP = torch.zeros_like(Pspec)
    _reaches(plan, "tvolap_adjoint_mac", lambda: plan.adjoint_mac(G, 0, X, 0, Pspec, 0, nb, dP))
    _refused(plan, lambda: plan.adjoint_mac(G, 0, X, 0, Pspec, 0, nb, dP[:, :pb - 1]))
    _refused(plan, lambda: plan.adjoint_mac(G[:N_OUT - 1], 0, X, 0, Pspec, 0, nb, dP))
    _reaches(plan, "tvolap_adjoint_mac_x", lambda: plan.adjoint_mac_x(G, 0, x, Pspec, 0, nb, dP))
    _refused(plan, lambda: plan.adjoint_mac_x(G, 0, g, Pspec, 0, nb, dP))
    _refused(plan, lambda: plan.adjoint_mac_x(G, 0, x, Pspec, 0, nb, dP,
                                              dX=z((N_OUT, nb, P), F32)), (ValueError, TypeError))
    _reaches(plan, "tvolap_adjoint_input", lambda: plan.adjoint_input(G, 0, x.clone()))
    _refused(plan, lambda: plan.adjoint_input(G, 0, g.clone()))


def test_nonuniform_block_extents():
    nu = object.__new__(NonUniform)
    nu.n_in, nu.n_out, nu.La = N_IN, N_OUT, L
    nu.device = torch.device("cpu")
    _recorder(nu)
    x = z((N_IN, L))
    _reaches(nu, "tvolap_nu_process_block", lambda: nu.process_block(x, z((N_OUT, L))))
    _refused(nu, lambda: nu.process_block(x, z((N_OUT, L - 1))))
    _refused(nu, lambda: nu.process_block(x, None, z(N_OUT - 1, I32)))
    _refused(nu, lambda: nu.process_signal(z((N_IN + 1, 64)), z((N_OUT, 8), I32)))
    sched = z((N_OUT, n_blocks_for(64, L)), I32)
    _reaches(nu, "tvolap_nu_process_signal", lambda: nu.process_signal(z((N_IN, 64)), sched))
    _reaches(nu, "tvolap_nu_process_signal",
             lambda: nu.process_signal(z((N_IN, 64)), sched, out=z((N_OUT, 70))))
    _refused(nu, lambda: nu.process_signal(z((N_IN, 64)), sched, out=z((N_OUT, 63))))
    _refused(nu, lambda: nu.process_signal(z((N_IN, 64)), sched, out=z((N_OUT - 1, 64))))


def test_batch_source_and_server_snapshot_buffers():
    b = object.__new__(BatchedTvolap)
    b.sources = [types.SimpleNamespace(x=np.zeros(100, np.float32), out_len=100, L=16)]
    b.device = torch.device("cuda", 0)
    b.h = None
    _recorder(b)
    _refused(b, lambda: b.set_source(0, z(100), z(8, I32)))            # host tensors
    _refused(b, lambda: b.set_source(1, z(100), z(8, I32)), IndexError)
    s = object.__new__(Server)
    _recorder(s)
    _refused(s, lambda: s.restore(z(4096)))                             # not a byte buffer
