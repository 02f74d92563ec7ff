"""Tensor-core complex products (pt_complex_product) against exact complex128 products.

The ACE contractions (M = Psi^H W, xi = W L^{-H}, xi^H X, xi Z) and the PT
projection (S = Psi^H H Psi, H Psi - Psi S; Alg. 3) of the mixed-precision path
run as 3xTF32 tensor-core products with FP32 accumulation. Each case draws
seeded complex64 operands, forms the exact product of those same complex64
values in complex128 with numpy (a library matmul), and bounds
max |C_gpu - C_exact| / max |C_exact|. Bound: 1e-5. Splitting each operand into
two TF32 parts keeps about 22 significant bits per product term (2^-22 ~ 2.4e-7).
The tensor core's FP32 accumulator truncates, so its error grows linearly with
the MMAs added into it (4.4e-5 after 2250 MMAs, measured); the kernel starts a
fresh accumulator every 48 MMAs and sums the windows in round-to-nearest FP32,
which leaves ~1e-6 (about what sequential FP32 FMAs give). Single-pass TF32
would give ~3e-4 and fails the bound.
Shapes cover all four op combinations, ragged tiles in M, N and K, split-K, the
triangular-B option, complex alpha and beta, and K = 0.
"""
import os

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def pkg():
    import paper_1905_01348_gb300 as p
    from paper_1905_01348_gb300 import build as b
    if not os.path.exists(p._native.LIB_PATH):
        b.build()
    p.load()
    return p


def c64(shape, seed):
    return syn.gaussian_vectors(shape, seed).astype(np.complex64)


def run(pkg, op_a, op_b, M, N, K, alpha=1.0, beta=0.0, upper_b=False, ws_mb=64, seed=0):
    import torch
    # column-major storage: a (rows x cols) matrix is a numpy array of shape (cols, rows)
    a_rows, a_cols = (M, K) if op_a == 0 else (K, M)
    b_rows, b_cols = (K, N) if op_b == 0 else (N, K)
    A = c64((a_cols, a_rows), seed)
    B = c64((b_cols, b_rows), seed + 1)
    opA = A.T if op_a == 0 else A.conj()                  # (M, K)
    opB = B.T if op_b == 0 else B.conj()                  # (K, N)
    if upper_b:
        opB = np.triu(opB)
        B = (opB.T if op_b == 0 else opB.conj()).astype(np.complex64)
        opB = B.T if op_b == 0 else B.conj()
    C0 = syn.gaussian_vectors((N, M), seed + 2)           # column-major M x N, complex128
    exact = alpha * (opA.astype(np.complex128) @ opB.astype(np.complex128)) + beta * C0.T
    dev = "cuda:0"
    dA = torch.from_numpy(np.ascontiguousarray(A)).to(dev)
    dB = torch.from_numpy(np.ascontiguousarray(B)).to(dev)
    dC = torch.from_numpy(np.ascontiguousarray(C0)).to(dev)
    ws = torch.empty(max(ws_mb << 20, 256), dtype=torch.uint8, device=dev)   # 256 bytes: status word only
    stream = torch.cuda.current_stream().cuda_stream
    pkg.pt_complex_product(op_a, op_b, M, N, K, alpha, dA.data_ptr(), max(a_rows, 1), dB.data_ptr(), max(b_rows, 1),
                           beta, dC.data_ptr(), max(M, 1), upper_b, ws.data_ptr(), ws.numel(), stream)
    got = dC.cpu().numpy().T
    scale = max(np.max(np.abs(exact)), 1e-300)
    return float(np.max(np.abs(got - exact)) / scale)


@pytest.mark.parametrize("op_a,op_b,M,N,K", [
    (1, 0, 200, 150, 5003),      # A^H B, split-K, ragged everywhere
    (1, 0, 432, 432, 4001),      # the ACE / projection shape with a shorter basis
    (0, 0, 1000, 130, 77),       # -xi Z and H Psi - Psi S shape
    (0, 1, 300, 70, 70),
    (1, 1, 150, 140, 2000),
    (1, 0, 1, 1, 1),
    (0, 0, 129, 129, 9),
])
def test_product_matches_exact(pkg, op_a, op_b, M, N, K):
    assert run(pkg, op_a, op_b, M, N, K) < TOL


def test_alpha_beta_and_no_split(pkg):
    assert run(pkg, 1, 0, 260, 190, 3000, alpha=-0.5 + 2.0j, beta=0.25 - 1.0j) < TOL
    # no room for partials: the reduction runs unsplit (one accumulator per tile over all of K)
    assert run(pkg, 1, 0, 260, 190, 3000, alpha=1.0, beta=1.0, ws_mb=0) < TOL
    assert run(pkg, 1, 0, 130, 130, 20000, ws_mb=0) < TOL


def test_upper_triangular_b(pkg):
    assert run(pkg, 0, 1, 700, 300, 300, upper_b=True) < TOL
    assert run(pkg, 0, 0, 700, 300, 300, upper_b=True, alpha=-1.0, beta=1.0) < TOL


def test_empty_reduction_scales_c(pkg):
    assert run(pkg, 1, 0, 50, 40, 0, alpha=1.0, beta=2.0 - 1.0j) < 1e-14
