"""The allocation-free exponential entry point agrees with the allocating one (GPU).

etp_expm_e1_noalloc serves callers that cannot allocate device memory (for
example real-time loops where cudaMalloc could stall the device, or hosts whose
device memory comes from another allocator as fixed buffers): they pass device
buffers for H and the result, and the workspace is a static device array.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_expm_matches_allocating_entry_point():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2405_05213_gb300 import etp
    assert torch.cuda.is_available()
    ctx = etp.Context(0)
    rng = np.random.default_rng(7)
    # two calls in a row (different sizes, so stale workspace from the first
    # call overlaps the second one's matrices)
    for n, scale, tau in [(64, 30.0, 0.7), (23, 4.0, 1.3)]:
        H = np.triu(rng.standard_normal((n, n)), -1) * scale / np.sqrt(n)
        ref = etp.etp_expm_e1(ctx.h, H, tau)
        H_dev = torch.from_numpy(np.asfortranarray(H).ravel(order="F").copy()).cuda()
        y_dev = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        etp.etp_expm_e1_noalloc(ctx.h, n, H_dev, tau, y_dev)
        y = y_dev.cpu().numpy()
        assert np.all(np.isfinite(y))
        assert rel(y, ref) < 1e-12, (n, rel(y, ref))
    # sizes beyond the static workspace are rejected with a clear error
    H = torch.zeros(65 * 65, dtype=torch.float64, device="cuda")
    y = torch.zeros(65, dtype=torch.float64, device="cuda")
    with pytest.raises(etp.EtpError, match="1..64"):
        etp.etp_expm_e1_noalloc(ctx.h, 65, H, 0.5, y)
