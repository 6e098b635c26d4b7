"""The 3xTF32 tensor-core GEMM (tcgen05.mma kind::tf32 with the operands
split into TF32 head and tail) that the mixed form uses for the products
of Eq. (tmat) / Eq. (schurmat) of large boxes, through the C ABI.

* Small integers are exact in TF32 and their products and sums exact in
  FP32, so C - A B must come out exactly: any error in the shared-memory
  layout, the descriptors or the tensor-memory read-back shows as a wrong
  entry.
* Random FP64 operands: every entry within K 2^-22 (|A| |B|) of the FP64
  product (FP32 accuracy), which a single TF32 product (2^-11) misses.
Shapes cover one tile, ragged edges in M, N and K, and several tiles."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _colmajor(a):
    import torch
    a = np.asarray(a, dtype=np.float64)
    return torch.tensor(a.T.copy(), device="cuda").t()


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (128, 128, 8),
                                   (77, 50, 13), (300, 200, 97),
                                   (513, 257, 600)])
def test_integer_operands_are_exact(M, N, K):
    import paper_2001_11619_gb300 as skel
    rng = np.random.default_rng(M + N + K)
    A = rng.integers(-20, 21, (M, K)).astype(np.float64)
    B = rng.integers(-20, 21, (K, N)).astype(np.float64)
    C = rng.integers(-1000, 1001, (M, N)).astype(np.float64)
    c = _colmajor(C)
    skel.gemm_tf32x3(_colmajor(A), _colmajor(B), c)
    assert np.array_equal(c.cpu().numpy(), C - A @ B)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (200, 333, 450),
                                   (1000, 700, 1300)])
def test_random_operands_reach_fp32_accuracy(M, N, K):
    import paper_2001_11619_gb300 as skel
    rng = np.random.default_rng(7 * M + N)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, (M, 1)))
    B = rng.standard_normal((K, N))
    C = rng.standard_normal((M, N))
    c = _colmajor(C)
    skel.gemm_tf32x3(_colmajor(A), _colmajor(B), c)
    err = np.abs(c.cpu().numpy() - (C - A @ B))
    scale = np.abs(A) @ np.abs(B)
    ratio = (err / scale).max()
    assert ratio < K * 2.0 ** -22
    assert ratio < 2.0 ** -14   # far below one TF32 product's 2^-11


def test_rejects_bad_strides():
    import paper_2001_11619_gb300 as skel
    import torch
    a = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        skel.gemm_tf32x3(a, a, a)   # row-major


def test_mixed_form_with_tensor_core_products_meets_the_target():
    """The mixed form with the wide boxes' products of Eq. (tmat) /
    Eq. (schurmat) on the tensor cores (tc_products, wide boxes from 200
    active DOFs) on the clustered-hole case: the preconditioner is weaker
    but GMRES reaches the same backward error and forward error against
    the dense LU as the FP64-product run."""
    import oracle
    import paper_2001_11619_gb300 as skel
    from gpu_util import assert_solution_close, solver
    from test_gpu_parity_paths import backward_error, quad_holes32
    wl = quad_holes32()
    g = oracle.quadrature(wl)
    A = oracle.dense_system(g)
    f = oracle.boundary_data(g, wl.src_xy[:1], wl.src_f[:1])
    x = np.linalg.solve(A, f)
    s = solver(wl, precision=skel.MIXED, id_tol=1e-6, gmres_tol=1e-12,
               gmres_maxit=120)
    s.set_tuning(wide_min_n=200, tc_products=1)
    s.factor()
    assert sum(lv["wide_boxes"] for lv in s.stats()["per_level"]) > 0
    xs = np.asarray(s.solve(f))
    assert backward_error(A, xs, f) < 1e-10
    assert_solution_close(xs, x, wl, 1e-8, "tensor-core products")
    s.close()
