"""The skinny Gram product (reorthogonalisation / Rayleigh-Ritz building block)
against numpy in FP64 on the same (rounded) fields: tiny, ragged and
tile-multiple lengths, aligned strides (TMA path) and packed odd strides
(plain path), every row/column count class and lane layout."""
import numpy as np
import pytest
import torch

import inputs
from oracle.model import Model
from gpu_util import context, require_gpu, to_np

pytestmark = pytest.mark.gpu

FULL = dict(J=(1.0, -0.1, -0.05), D=0.3, K=0.05, muB=0.02)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 2e-6)])
@pytest.mark.parametrize("L1,L2", [(7, 6), (37, 29), (64, 64), (160, 97)])
@pytest.mark.parametrize("aligned", [True, False])
def test_gram_matches_numpy(dtype, tol, L1, L2, aligned):
    require_gpu()
    import paper_2509_26269_gb300 as mo
    ctx = context(Model(L1, L2, **FULL), dtype)
    n = 3 * L1 * L2
    ld = (n + 63) // 64 * 64 if aligned else n
    rng = inputs.normal(L1 * 100 + L2, 104 * ld).reshape(104, ld)
    buf = torch.from_numpy(rng).to(device="cuda", dtype=dtype)
    A = to_np(buf)[:, :n]
    # every lane-layout class of the streaming kernel (field counts rounded
    # up to 8: 8 ... 96) and the row sizes 1 KB (<= 32), 512 B (<= 72), 256 B
    for nx, ny in [(1, 1), (3, 3), (8, 8), (9, 3), (24, 8), (32, 8), (40, 5), (48, 8), (53, 8), (61, 1), (72, 8),
                   (80, 2), (88, 8), (96, 8)]:
        out = torch.empty(nx * ny, dtype=torch.float64, device="cuda")
        X = buf[0:nx].contiguous() if not aligned else buf
        Y = buf[nx:nx + ny]
        mo.moto_gram(ctx.handle, buf.data_ptr(), ld, nx, buf[nx].data_ptr() if ny else 0, ld, ny, out)
        ref = A[:nx] @ A[nx:nx + ny].T
        scale = np.abs(A[:nx]) @ np.abs(A[nx:nx + ny]).T
        err = np.abs(to_np(out).reshape(nx, ny) - ref) / scale
        assert err.max() <= tol, (nx, ny, err.max())
    ctx.close()
