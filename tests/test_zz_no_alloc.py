"""vlbm_diagnostics_noalloc: the diagnostics of a caller-owned device array for
callers that cannot call cudaMalloc where they need the numbers (their own
memory pools or budgets, latency-bound loops).  Its output must agree with
vlbm_diagnostics on the same populations, on two calls in a row (the shared
scratch keeps the last call's contents), count the cells that hold a NaN or Inf,
and refuse grids beyond its fixed scratch size.

This file is named to be collected last."""
import numpy as np
import pytest

from parity import require_gpu
from paper_2504_15574_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_noalloc_diagnostics_match_the_allocating_entry_point():
    require_gpu()
    import torch

    from paper_2504_15574_gb300 import build, vlbm
    build.build()
    vlbm.load()
    keys = ["mass", "px", "py", "pz", "energy"]
    for (nt, np_, run) in [(24, 48, 1), (13, 10, 2)]:
        s = vlbm.Solver(nt, np_, 0.02, 1e-4)
        s.init_moments(*inputs.gaussian_vortices(nt, np_, run=run))
        s.step(3)
        ref = s.diagnostics()
        f = s.get_populations()
        s.close()
        f_dev = torch.from_numpy(f).to("cuda")
        for call in range(2):
            out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
            vlbm.vlbm_diagnostics_noalloc(f_dev.data_ptr(), nt, np_, 1.0, out.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            for q, k in enumerate(keys):
                assert got[q] == pytest.approx(ref[k], rel=1e-12, abs=1e-14 * ref["mass"]), (call, k)
            assert got[5] == 0.0


def test_noalloc_rejects_grids_beyond_its_scratch():
    require_gpu()
    import torch

    from paper_2504_15574_gb300 import vlbm
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    f = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(vlbm.VlbmError) as e:
        vlbm.load()
        vlbm.vlbm_diagnostics_noalloc(f.data_ptr(), 16385, 2, 1.0, out.data_ptr())
    assert e.value.code == vlbm.VLBM_ERR_ARG
    assert "16384" in str(e.value)


def test_noalloc_counts_the_cells_holding_a_nonfinite_population():
    require_gpu()
    import torch

    from paper_2504_15574_gb300 import vlbm
    vlbm.load()
    nt, np_ = 12, 16
    s = vlbm.Solver(nt, np_, 0.02, 1e-4)
    s.init_moments(*inputs.gaussian_vortices(nt, np_, run=4))
    f = s.get_populations()
    s.close()
    # two cells of row 3 (one with two bad populations), one cell of row 9 (an infinity)
    f[2, 3, 5] = np.nan
    f[7, 3, 5] = np.nan
    f[11, 3, 6] = np.nan
    f[0, 9, 0] = np.inf
    f_dev = torch.from_numpy(f).to("cuda")
    for call in range(2):
        out = torch.zeros(6, dtype=torch.float64, device="cuda")
        vlbm.vlbm_diagnostics_noalloc(f_dev.data_ptr(), nt, np_, 1.0, out.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert out[5].item() == 3.0, (call, out[5].item())
