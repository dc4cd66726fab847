"""mt_transfer_1d_noalloc: the entry point for callers that cannot allocate
device memory (so cannot hand libmt a workspace).  Its intermediates live in
a fixed array inside the library; this checks that it gives the same masses
as the workspace-based step, on two calls in a row, through the C ABI, under
both normalisations and with and without the reaction, and that it refuses
inputs it cannot handle.

Kept in its own file, collected last, so that a failure here does not stop
the rest of the GPU suite."""
import numpy as np
import pytest

from paper_1811_05474_gb300 import mt, synth

pytestmark = pytest.mark.gpu


def _call(xs, a, b, ao, bo, n, L, norm=mt.MT_NORM_SYM, react=1):
    mt.mt_transfer_1d_noalloc(xs.data_ptr(), a.data_ptr(), b.data_ptr(), ao.data_ptr(),
                              bo.data_ptr(), n, L, 0.1, 1.0, 0.0, norm, react, None)


@pytest.mark.parametrize("norm", [mt.MT_NORM_SYM, mt.MT_NORM_ROW])
@pytest.mark.parametrize("react", [1, 0])
def test_noalloc_matches_workspace_step_on_two_calls(norm, react):
    import torch

    n, L = 60000, 60000.0
    x = synth.uniform_positions(n, L, seed=71)
    A, B = synth.uniform_masses(n, seed=71)
    # existing entry point: two steps with no random walk, binary64
    p = mt.mt_params_init(n=n, L=(L,), D_rw=0.0, precision=mt.MT_FP64, norm=norm, react=react)
    sim = mt.Simulation(p)
    sim.upload(x, A, B)
    ref = []
    for _ in range(2):
        sim.step()
        ref.append(sim.masses())
    sim.close()
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
        _call(xs, a, b, ao, bo, n, L, norm, react)
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


@pytest.mark.parametrize("case", ["beyond_L", "negative", "nan", "reversed", "one_swap"])
def test_noalloc_rejects_bad_positions(case):
    """Positions outside [0, L], NaN, or out of ascending order: MT_ERR_INVALID
    (the outputs are undefined then).  Reversed positions make every walk
    stop at its first neighbour, so the rejected call stays cheap."""
    import torch

    n, L = 4096, 4096.0
    x = np.sort(synth.uniform_positions(n, L, seed=5)[0])
    if case == "beyond_L":
        x[-1] = L + 1.0
    elif case == "negative":
        x[0] = -0.5
    elif case == "nan":
        x[n // 2] = np.nan
    elif case == "reversed":
        x = x[::-1].copy()
    else:
        x[100], x[101] = x[101], x[100] - 1e-3
    A, B = synth.uniform_masses(n, seed=5)
    dev = torch.device("cuda")
    xs, a, b = (torch.tensor(v, device=dev) for v in (x, A, B))
    ao, bo = torch.empty_like(a), torch.empty_like(b)
    with pytest.raises(mt.MtError) as e:
        _call(xs, a, b, ao, bo, n, L)
    assert e.value.status == mt.MT_ERR_INVALID
    # the library stays usable: a good call right after succeeds
    xs = torch.tensor(np.sort(synth.uniform_positions(n, L, seed=6)[0]), device=dev)
    _call(xs, a, b, ao, bo, n, L)
    torch.cuda.synchronize()


def test_noalloc_empty_input_is_a_no_op():
    mt.mt_transfer_1d_noalloc(None, None, None, None, None, 0, 10.0, 0.1, 1.0, 0.0,
                              mt.MT_NORM_SYM, 1, None)
