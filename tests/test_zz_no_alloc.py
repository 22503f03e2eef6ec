"""GPU test of rbc_nusselt_static, the entry point that allocates no device memory.

Some callers cannot allocate device memory when they ask for a diagnostic: an
application whose pool allocator already holds the free device memory, or a
timed loop that cannot pay for the synchronisation cudaMalloc/cudaFree may
cause.  rbc_nusselt_static serves them with scratch in a fixed device array of
the library.  This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _static_nusselt(rbc, F, state):
    out = np.zeros(3)
    st = rbc.load().rbc_nusselt_static(F.h, ctypes.c_void_p(state.data_ptr()),
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


def test_static_scratch_nusselt_matches_rbc_nusselt_on_consecutive_calls():
    from paper_2001_01609_gb300 import build
    build.build()
    from paper_2001_01609_gb300 import rbc
    from paper_2001_01609_gb300.inputs import initial_temperature

    assert torch.cuda.is_available()
    for (Nx, Nz, Ra) in ((64, 32, 1e5), (256, 64, 1e6)):
        F = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, 1e-5)
        st = F.new_states(2)
        for b in range(2):
            F.set_state(st[b], initial_temperature(Nx, Nz, seed=10 + b, amplitude=0.3))
        F.step_batch(st, 3)
        for b in (0, 1, 0, 1):                         # two calls in a row per state, states alternating
            ref = np.array(F.nusselt(st[b]))           # the allocating entry point
            for _ in range(2):
                status, out = _static_nusselt(rbc, F, st[b])
                assert status == rbc.RBC_OK
                np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-13)


def test_static_scratch_nusselt_on_a_fresh_mixed_precision_handle_allocates_nothing():
    """A mixed-precision handle on a grid of 64 Chebyshev coefficients runs the
    tensor-core z-inverse, whose bounded
    waits report through an error word: the call keeps that word in the static
    array too.  The handle is fresh (it never reserved a workspace) and the
    device's free memory does not change across the calls."""
    from paper_2001_01609_gb300 import build
    build.build()
    from paper_2001_01609_gb300 import rbc
    from paper_2001_01609_gb300.inputs import initial_temperature

    Nx, Nz, Ra = 64, 64, 1e5
    prep = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, 1e-5, precision=rbc.RBC_MIXED)
    st = prep.new_states(2)
    for b in range(2):
        prep.set_state(st[b], initial_temperature(Nx, Nz, seed=20 + b, amplitude=0.3))
    prep.step_batch(st, 3)
    refs = [np.array(prep.nusselt(st[b])) for b in range(2)]   # the allocating entry point
    status, _ = _static_nusselt(rbc, prep, st[0])               # module and array loaded before measuring
    assert status == rbc.RBC_OK
    fresh = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, 1e-5, precision=rbc.RBC_MIXED)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for b in (0, 1):
        for _ in range(2):                                      # two calls in a row
            status, out = _static_nusselt(rbc, fresh, st[b])
            assert status == rbc.RBC_OK
            np.testing.assert_allclose(out, refs[b], rtol=1e-12, atol=1e-13)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_scratch_nusselt_rejects_grids_beyond_its_size():
    from paper_2001_01609_gb300 import rbc

    F = rbc.Propagator(1e6, 1.0, 2.0, 256, 128, 1e-5)
    st = F.new_states(1)
    status, out = _static_nusselt(rbc, F, st[0])
    assert status == rbc.RBC_EINVAL
    assert b"static array" in rbc.load().rbc_last_error()
