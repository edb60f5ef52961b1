"""trtr_phi_sums_noalloc, the entry point for callers that cannot allocate device memory
(their HBM belongs to another allocator, cudaMalloc's implicit synchronisation is not
acceptable in their loop, or their host forbids libraries from allocating).

It must give the same mass and error sums as the context-based reductions (trtr_mass,
trtr_error_vs) on the same populations, on two calls in a row through the shared static
scratch array.  This file is collected last so that a run stopping at the first failure
has already run every other test; it also passes on its own in a fresh process.
"""
import math

import numpy as np
import pytest

from paper_2312_10316_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2312_10316_gb300 import trtr as T  # noqa: E402

REL_TOL = 1e-12  # both sides sum the same FP64 values, in different orders


@pytest.mark.parametrize("precision", [T.TRTR_F64, T.TRTR_F32])
def test_noalloc_sums_match_context_reductions_twice(precision):
    pulse = W.Pulse(n=200, D_amp=0.5, courant=0.8, D0=0.2766 / 3 * (2 / 200) ** 2 / W.Pulse(n=200, courant=0.8).dt)
    nx = ny = pulse.n
    stream = torch.cuda.Stream()
    with T.pulse_solver(pulse, precision=precision, stream=stream.cuda_stream) as s:
        s.step(40)
        g = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
        s.get_populations(g)
        ref_np = W.phi_analytic(pulse, 40 * pulse.dt)
        ref = torch.from_numpy(ref_np).cuda()
        mass_ctx = s.mass()
        rms_ctx, rel_ctx = s.error_vs(ref_np)
        for call in range(2):
            out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            st = T.trtr_phi_sums_noalloc(g, nx, ny, ref, out, stream.cuda_stream)
            assert st == T.TRTR_OK, T.trtr_status_str(st)
            stream.synchronize()
            a, b, c = out.cpu().numpy()
            assert abs(a - mass_ctx) <= REL_TOL * abs(mass_ctx), (call, a, mass_ctx)
            assert abs(math.sqrt(b / (nx * ny)) - rms_ctx) <= REL_TOL * rms_ctx, call
            assert abs(math.sqrt(b / c) - rel_ctx) <= REL_TOL * rel_ctx, call
        # without a reference field only the mass is formed
        out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        assert T.trtr_phi_sums_noalloc(g, nx, ny, None, out, stream.cuda_stream) == T.TRTR_OK
        stream.synchronize()
        a, b, c = out.cpu().numpy()
        assert abs(a - mass_ctx) <= REL_TOL * abs(mass_ctx) and b == 0.0 and c == 0.0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    g = torch.zeros(9 * 4, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    rows = 16385  # TRTR_NOALLOC_MAX_ROWS + 1
    big = torch.zeros(9 * rows, dtype=torch.float64, device="cuda")
    assert T.trtr_phi_sums_noalloc(big, 1, rows, None, out, None) == T.TRTR_EINVAL
    assert T.trtr_phi_sums_noalloc(g, 0, 4, None, out, None) == T.TRTR_EINVAL
    assert T.lib.trtr_phi_sums_noalloc(None, 2, 2, None, out.data_ptr(), None) == T.TRTR_EINVAL
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), np.zeros(3))
