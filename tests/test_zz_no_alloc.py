"""pp_orthogonalize_noalloc against pp_orthogonalize, through the C-ABI.

pp_orthogonalize_noalloc is for callers that cannot allocate device memory
(their GPU memory is reserved by another framework's allocator, or their loop
cannot afford cudaMalloc's possible device synchronisation): it runs the same
CGS2 step with the caller's buffers and a fixed scratch array compiled into the
library.  Two calls in a row, each compared with the allocating entry point on
identical inputs, within the tolerance of the CGS2 parity test
(test_orthogonalize_matches_oracle_cgs2: 4 n u ||w|| per coefficient).
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1806_08020_gb300 import inputs

pytestmark = pytest.mark.gpu

U = np.finfo(np.float64).eps / 2


def test_noalloc_matches_allocating_entry_point():
    import torch
    from paper_1806_08020_gb300 import pp
    stream = torch.cuda.current_stream().cuda_stream
    for n, j in ((100003, 51), (4099, 128)):  # two calls in a row
        rng = np.random.default_rng(n + j)
        Q, _ = np.linalg.qr(rng.standard_normal((n, j)))
        w = rng.standard_normal(n) + Q @ rng.standard_normal(j) * 10
        ldv = (n + 31) // 32 * 32
        Vd = torch.zeros((j, ldv), dtype=torch.float64, device="cuda")
        Vd[:, :n] = torch.tensor(Q.T)
        # allocating entry point (through a context)
        ctx = pp.pp_create(inputs.diagonal(np.ones(n)), stream=stream)
        w_ref = torch.tensor(w, device="cuda")
        v_ref = torch.empty(n, dtype=torch.float64, device="cuda")
        h_ref = pp.pp_orthogonalize(ctx, Vd.data_ptr(), ldv, j, w_ref.data_ptr(), v_ref.data_ptr())
        # allocation-free entry point, caller-owned buffers only
        w_na = torch.tensor(w, device="cuda")
        v_na = torch.empty(n, dtype=torch.float64, device="cuda")
        h_na = torch.empty(j + 1, dtype=torch.float64, device="cuda")
        pp.pp_orthogonalize_noalloc(n, Vd.data_ptr(), ldv, j, w_na.data_ptr(), v_na.data_ptr(), h_na.data_ptr(),
                                    stream)
        torch.cuda.synchronize()
        tol = 4 * n * U * np.linalg.norm(w)
        h = h_na.cpu().numpy()
        assert np.abs(h - h_ref).max() <= tol
        assert np.abs(v_na.cpu().numpy() - v_ref.cpu().numpy()).max() <= 4 * tol / h_ref[j]
        assert np.abs(w_na.cpu().numpy() - w_ref.cpu().numpy()).max() <= tol
        assert np.abs(Q.T @ v_na.cpu().numpy()).max() <= 1e-12 * np.sqrt(n)
        ctx.close()
    # sizes beyond the static scratch are rejected with a clear error
    with pytest.raises(pp.PPError, match="outside"):
        pp.pp_orthogonalize_noalloc(1000, Vd.data_ptr(), 1024, 129, w_na.data_ptr(), v_na.data_ptr(),
                                    h_na.data_ptr(), stream)
