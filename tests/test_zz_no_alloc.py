"""mt_transfer_1d_noalloc: the entry point for callers that cannot allocate
device memory (so cannot hand libmt a workspace).  Its intermediates live in
a fixed array inside the library; this checks that it gives the same masses
as the workspace-based step, on two calls in a row, through the C ABI.

Kept in its own file, collected last, so that a failure here does not stop
the rest of the GPU suite."""
import numpy as np
import pytest

from paper_1811_05474_gb300 import mt, synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_workspace_step_on_two_calls():
    import torch

    n, L = 60000, 60000.0
    x = synth.uniform_positions(n, L, seed=71)
    A, B = synth.uniform_masses(n, seed=71)
    # existing entry point: two steps with no random walk, binary64
    p = mt.mt_params_init(n=n, L=(L,), D_rw=0.0, precision=mt.MT_FP64)
    sim = mt.Simulation(p)
    sim.upload(x, A, B)
    ref = []
    for _ in range(2):
        sim.step()
        ref.append(sim.masses())
    # new entry point on the same particles, sorted by position
    order = np.argsort(x[0], kind="stable")
    dev = torch.device("cuda")
    xs = torch.tensor(x[0][order], device=dev)
    a = torch.tensor(A[order], device=dev)
    b = torch.tensor(B[order], device=dev)
    torch.cuda.synchronize()
    for call in range(2):
        ao = torch.empty_like(a)
        bo = torch.empty_like(b)
        mt.mt_transfer_1d_noalloc(xs.data_ptr(), a.data_ptr(), b.data_ptr(), ao.data_ptr(),
                                  bo.data_ptr(), n, L, 0.1, 1.0, 0.0, mt.MT_NORM_SYM, 1, None)
        ra, rb = ref[call]
        for got, want in ((ao.cpu().numpy(), ra[order]), (bo.cpu().numpy(), rb[order])):
            err = np.abs(got - want) / np.maximum(np.abs(want), 0.5)
            assert err.max() <= 1e-12, f"call {call}: max rel err {err.max():.3e}"
        a, b = ao, bo


def test_noalloc_rejects_sizes_beyond_its_scratch():
    with pytest.raises(mt.MtError) as e:
        mt.mt_transfer_1d_noalloc(None, None, None, None, None, (1 << 20) + 1, 10.0, 0.1, 1.0,
                                  0.0, mt.MT_NORM_SYM, 1, None)
    assert e.value.status == mt.MT_ERR_INVALID
    assert "1048576" in mt.mt_last_error()
