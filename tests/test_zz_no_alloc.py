"""gabp_run_rounds_noalloc: FP64 rounds whose working space is a fixed static
device array, for callers that cannot allocate device memory when they call
(applications that reserve all device memory up front, code inside an
allocator callback, loops that must not synchronise the device through
cudaMalloc/cudaFree).

Checked through the C ABI against the oracle's synchronous rounds
(Algorithm 2) and against gabp_run_rounds (the handle-based entry point,
which allocates its message buffers) on two calls in a row, within the 1e-12
relative tolerance of the FP64 round parity tests; and checked to leave the
device's free memory and the caching allocator's reservation unchanged on
repeated calls.  This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes on its own in
a fresh process.
"""
import numpy as np
import pytest

import oracle
from paper_0810_1119_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU hosts
    pytest.skip("CUDA device required", allow_module_level=True)


@pytest.fixture(scope="module")
def G():
    from paper_0810_1119_gb300 import build_lib
    build_lib.build()
    from paper_0810_1119_gb300 import gabp
    gabp.load()
    return gabp


def _rel(a, ref):
    return float(np.abs(a - ref).max() / max(np.abs(ref).max(), 1e-300))


def _device_csr(m):
    dev = "cuda"
    return (torch.tensor(m.row_ptr, dtype=torch.int64, device=dev),
            torch.tensor(m.col, dtype=torch.int32, device=dev),
            torch.tensor(m.val, dtype=torch.float64, device=dev),
            torch.tensor(W.reverse_index(m), dtype=torch.int64, device=dev))


def test_noalloc_rounds_match_handle_rounds_twice(G):
    m = W.er_sdd(9000, 8, 1.1, 21)                 # ~81k entries, within the 2^18 limit
    rp, cl, vl, rv = _device_csr(m)
    ref_handle = G.Solver.from_csr(m.row_ptr, m.col, m.val)
    for call, (seed, rounds) in enumerate(((1, 7), (2, 12))):
        b = torch.tensor(W.normal_rhs(m.n, seed), device="cuda")
        x_noalloc = torch.full_like(b, float("nan"))
        G.gabp_run_rounds_noalloc(rp, cl, vl, rv, b, rounds, x_noalloc)
        x_ref = torch.empty_like(b)
        G.gabp_run_rounds(ref_handle.handle, b, rounds, x_ref)
        err = _rel(x_noalloc.cpu().numpy(), x_ref.cpu().numpy())
        assert err <= 1e-12, (call, err)
    ref_handle.close()


@pytest.mark.parametrize("rounds", [0, 1, 7, 12])
def test_noalloc_rounds_match_the_oracle(G, rounds):
    # Tentative means after `rounds` rounds from zero messages; rounds = 0
    # gives b_i / A_ii.  Two graphs: a random loopy one and an indefinite tree.
    for m, seed in ((W.er_sdd(3000, 8, 1.1, 31), 5),
                    (W.random_tree(400, 3, diag_scale=1.0, indefinite=True), 6)):
        rp, cl, vl, rv = _device_csr(m)
        b_h = W.normal_rhs(m.n, seed)
        x = torch.full((m.n,), float("nan"), dtype=torch.float64, device="cuda")
        G.gabp_run_rounds_noalloc(rp, cl, vl, rv, torch.tensor(b_h, device="cuda"), rounds, x)
        ref = oracle.gabp(m.row_ptr, m.col, m.val, b_h, max_rounds=rounds)["x"]
        err = _rel(x.cpu().numpy(), ref)
        assert err <= 1e-12, (m.n, rounds, err)


def test_noalloc_repeated_calls_allocate_nothing(G):
    # After one call (which may load the library's module on this device),
    # further calls change neither the device's free memory (cudaMemGetInfo)
    # nor what torch's caching allocator holds.
    m = W.er_sdd(20000, 8, 1.1, 41)
    rp, cl, vl, rv = _device_csr(m)
    b = torch.tensor(W.normal_rhs(m.n, 3), device="cuda")
    x = torch.empty_like(b)
    G.gabp_run_rounds_noalloc(rp, cl, vl, rv, b, 5, x)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    allocated0 = torch.cuda.memory_allocated()
    for rounds in (5, 9, 3):
        G.gabp_run_rounds_noalloc(rp, cl, vl, rv, b, rounds, x)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_reserved() == reserved0
    assert torch.cuda.memory_allocated() == allocated0


def test_noalloc_rejects_matrices_beyond_its_fixed_space(G):
    m = W.poisson2d(300)                            # 448,800 entries > 2^18
    rp, cl, vl, rv = _device_csr(m)
    b = torch.ones(m.n, dtype=torch.float64, device="cuda")
    x = torch.empty_like(b)
    with pytest.raises(G.GabpError) as ei:
        G.gabp_run_rounds_noalloc(rp, cl, vl, rv, b, 3, x)
    assert ei.value.name == "GABP_ERR_INVALID_ARG"
    assert "262144" in str(ei.value)
