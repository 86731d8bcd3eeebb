"""The allocation-free step, lbm_step_fixed_scratch, against lbm_step.

Callers that cannot allocate device memory (a plugin inside a framework
that owns all allocations, a capped or exhausted allocator) step the
lattice through
lbm_step_fixed_scratch, which keeps its macroscopic record, ghost planes and
status word in a device array compiled into the library.  This test calls
it through the C ABI twice in a row and compares each output -- populations
and temperatures -- with what the context-based lbm_step produces from the
same state, using the double-precision parity tolerance (1e-10 of each
set's largest magnitude).

The file is named to be collected last, so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

import workload as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2101_01702_gb300 import build
    build.build()
    from paper_2101_01702_gb300 import lbm as L
    return L


def _current_state(solver, L):
    """The solver's current populations (double view) and its temperature row."""
    ptr = L.lbm_state_buffer(solver.ctx)
    buf = solver.pop[0] if solver.pop[0].data_ptr() == ptr else solver.pop[1]
    assert buf.data_ptr() == ptr
    return buf.view(dtype=__import__("torch").float64), solver.macro[: solver.N]


def _rel_per_set(got, ref, S):
    g = got.reshape(S, -1).double().cpu().numpy()
    r = ref.reshape(S, -1).double().cpu().numpy()
    return max(float(np.abs(g[s] - r[s]).max() / np.abs(r[s]).max()) for s in range(S))


@pytest.mark.parametrize("case", ["three_gas_periodic", "nine_species_ghost_nodes"])
def test_fixed_scratch_step_matches_lbm_step(lbm, case):
    import torch
    prob = w.config1_problem() if case == "three_gas_periodic" else w.flame1d_problem(nx=256)
    ref = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    stream = torch.cuda.current_stream().cuda_stream
    pop, T = _current_state(ref, lbm)
    pop_in = pop.clone()
    T_io = T.clone()
    for call in range(2):
        pop_out = torch.empty_like(pop_in)
        st = lbm.lbm_step_fixed_scratch(ref.lat, ref.sp, ref.mech, pop_in.data_ptr(), pop_out.data_ptr(),
                                        T_io.data_ptr(), stream)
        assert st == lbm.LBM_OK, lbm.lbm_strerror(st)
        ref.step(1)
        pop_ref, T_ref = _current_state(ref, lbm)
        torch.cuda.synchronize()
        assert _rel_per_set(pop_out, pop_ref, ref.S) <= 1e-10, call
        assert float(((T_io - T_ref).abs().max() / T_ref.abs().max()).item()) <= 1e-10, call
        pop_in = pop_out
    ref.close()


def test_fixed_scratch_rejects_lattices_beyond_the_array(lbm):
    import torch
    # the record takes (31 + 8 M) * 8 B per node: 44^3 nodes with M = 9 is the
    # first cube beyond the 64 MiB array (43^3 fits); rejected before any
    # device work, so the dummy buffers are never touched
    prob = w.sphere3d_problem(n=44, radius=5.0)
    ref = lbm.Solver(prob.lattice, prob.species, prob.mech, precision=lbm.LBM_FP64)
    dummy = torch.empty(16, dtype=torch.float64, device="cuda")
    dummy2 = torch.empty(16, dtype=torch.float64, device="cuda")
    dummy3 = torch.empty(16, dtype=torch.float64, device="cuda")
    st = lbm.lbm_step_fixed_scratch(ref.lat, ref.sp, ref.mech, dummy.data_ptr(), dummy2.data_ptr(),
                                    dummy3.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == lbm.LBM_ERR_ARG
    ref.close()


def test_fixed_scratch_rejects_overlapping_buffers(lbm):
    """The temperature row is copied into the array before the step and back
    after it; a T_io inside either population buffer, or population buffers
    that overlap, would corrupt the state, so the call refuses them before
    any device work."""
    import torch
    prob = w.config1_problem()
    ref = lbm.Solver.from_problem(prob, precision=lbm.LBM_FP64)
    stream = torch.cuda.current_stream().cuda_stream
    pop, T = _current_state(ref, lbm)
    n_pop = pop.numel()
    pop_in, pop_out = pop.clone(), torch.empty_like(pop)
    both = torch.empty(n_pop + ref.N, dtype=torch.float64, device="cuda")
    T_io = T.clone()
    bad = [(pop_in, pop_out, pop_in[5:5 + ref.N]),                 # T_io inside pop_in
           (pop_in, pop_out, pop_out[n_pop - ref.N // 2:]),        # T_io runs into pop_out's tail
           (both[:n_pop], both[ref.N:], T_io)]                     # population buffers overlap
    before = pop_in.clone()
    for a, b, t in bad:
        st = lbm.lbm_step_fixed_scratch(ref.lat, ref.sp, ref.mech, a.data_ptr(), b.data_ptr(), t.data_ptr(), stream)
        assert st == lbm.LBM_ERR_ARG
    torch.cuda.synchronize()
    assert torch.equal(pop_in, before)
    ref.close()
