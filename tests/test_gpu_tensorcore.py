"""The tensor-core GEMM of the shared-shape variant (tcgen05, 3xTF32) against
FP64 matrix products: C = A . B^T for full, ragged and split-K shapes.

Error bound: the 3xTF32 split drops the lo.lo product and truncates the lo
parts to TF32, about 2^-20 |a||b| per product, and the FP32 accumulation adds
about K 2^-24 sum |a b|; the test holds every element to
2e-6 (|A| |B|^T)_ij + 1e-30."""
import numpy as np
import pytest

from paper_2501_09308_gb300 import xrdvi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K,seed", [
    (128, 64, 32, 1),       # one tile, one k-block
    (200, 70, 56, 2),       # ragged rows and columns, partial last k-block
    (256, 500, 4608, 3),    # the backward's shape at the K=50 workload: split-K
    (1, 1, 4, 4),           # a single element
    (384, 64, 1024, 5),     # three row tiles, many k-blocks
])
def test_gemm_matches_fp64(M, N, K, seed):
    import torch
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, K)).astype(np.float32) * rng.uniform(0.5, 2.0, (M, 1)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    xrdvi.xrdvi_gemm_nt_tf32x3(M, N, K, dA.data_ptr(), K, dB.data_ptr(), K, dC.data_ptr(), N)
    C = dC.cpu().numpy().astype(np.float64)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    bound = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64)).T
    err = np.abs(C - ref)
    print(f"\nGEMM {M}x{N}x{K}: max err / (|A||B|^T) = {np.max(err / bound):.3e}")
    assert np.all(np.isfinite(C))
    assert np.all(err <= 2e-6 * bound + 1e-30)


def test_gemm_positive_operands_relative_accuracy():
    """Positive operands (the forward's intensities and phase profiles): the
    product is accurate to a few FP32 ulps relative."""
    import torch
    rng = np.random.default_rng(9)
    A = rng.uniform(0.0, 1.0, (256, 56)).astype(np.float32)
    B = rng.uniform(0.0, 3.0, (4608, 56)).astype(np.float32)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.empty((256, 4608), dtype=torch.float32, device="cuda")
    xrdvi.xrdvi_gemm_nt_tf32x3(256, 4608, 56, dA.data_ptr(), 56, dB.data_ptr(), 56, dC.data_ptr(), 4608)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    rel = np.max(np.abs(dC.cpu().numpy() - ref) / ref)
    print(f"\npositive 256x4608x56: max rel err {rel:.3e}")
    assert rel <= 2e-6


def test_gemm_rejects_unaligned_sizes():
    import torch
    d = torch.zeros(64, device="cuda")
    with pytest.raises(xrdvi.XrdviError) as e:
        xrdvi.xrdvi_gemm_nt_tf32x3(2, 2, 3, d.data_ptr(), 3, d.data_ptr(), 3, d.data_ptr(), 2)
    assert e.value.status == 1
