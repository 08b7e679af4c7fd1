"""The tensor-core tile GEMM building block (tcgen05.mma kind::f16, BF16
operands in 128-byte-swizzled shared memory, FP32 accumulation in TMEM)
against torch on the same BF16-rounded operands.  Shapes cover every
(N, K) the BF16 pair passes use: N in {16, 32, 48, 128, 176, 256}, K from 16
(one MMA) to 192 (three swizzle blocks) and the K = 176 partial block."""
import ctypes

import pytest
import torch

import paper_2303_08169_gb300 as al

pytestmark = pytest.mark.gpu


def _selftest(A, B):
    L = al.lib()
    fn = L.allegro_selftest_mma
    fn.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    N, K = B.shape
    D = torch.full((128, N), float("nan"), device="cuda")
    rc = fn(N, K, A.data_ptr(), B.data_ptr(), D.data_ptr())
    torch.cuda.synchronize()
    assert rc == 0, rc
    return D


@pytest.mark.parametrize("N,K", [(16, 16), (128, 16), (32, 128), (48, 128), (16, 128), (128, 128),
                                 (128, 176), (176, 128), (128, 192), (256, 64), (256, 256)])
def test_tile_gemm_matches_torch(N, K):
    g = torch.Generator(device="cuda").manual_seed(N * 1000 + K)
    A = torch.randn(128, K, device="cuda", generator=g)
    B = torch.randn(N, K, device="cuda", generator=g)
    D = _selftest(A, B)
    ref = A.bfloat16().double() @ B.bfloat16().double().T
    err = (D.double() - ref).abs().max().item()
    assert err <= 1e-5 * ref.abs().max().item() + 1e-5, err


@pytest.mark.parametrize("N,K", [(128, 128), (128, 32), (176, 128), (48, 16), (128, 48), (16, 128), (192, 64)])
def test_mn_major_b_operand(N, K):
    """d = a @ w with w (K x N) kept in its K-major image and read MN-major:
    the descriptor reading with lbo = K * 128 (stride between 64-column
    blocks) and sbo = 1024 (8 rows) must match torch; the exchanged reading is
    recorded but only one of the two can be right."""
    g = torch.Generator(device="cuda").manual_seed(7 * N + K)
    A = torch.randn(128, K, device="cuda", generator=g)
    W = torch.randn(K, N, device="cuda", generator=g)
    ref = A.bfloat16().double() @ W.bfloat16().double()
    D = torch.full((128, N), float("nan"), device="cuda")
    al.allegro_selftest_mma_mode(A, W, D, 1)
    torch.cuda.synchronize()
    err = (D.double() - ref).abs().max().item()
    assert err <= 1e-5 * ref.abs().max().item() + 1e-5, err


def test_silu_error_bound():
    """The error model of the tensor-core tests (tests/emulation_bounds.py)
    rests on this: the passes' SiLU, z sigmoid(z) with sigmoid through
    tanh.approx.f32, is within |z| 2^-17.5 of the exact value, and its
    derivative within (1 + |z|) 2^-17.5, on a dense grid over [-30, 30]
    (FP32 rounding of the final products added)."""
    x = torch.linspace(-30.0, 30.0, 1 << 22, device="cuda", dtype=torch.float32)
    y = torch.empty(2 * x.numel(), device="cuda", dtype=torch.float32)
    al.allegro_selftest_silu(x, y)
    z = x.double().cpu()
    s = torch.sigmoid(z)
    silu, dsilu = z * s, s * (1.0 + z * (1.0 - s))
    got = y.double().cpu().view(-1, 2)
    e1 = (got[:, 0] - silu).abs()
    e2 = (got[:, 1] - dsilu).abs()
    b = 2.0 ** -17.5
    assert bool((e1 <= z.abs() * b + 2.0 ** -23 * silu.abs()).all()), float((e1 / (z.abs() * b + 1e-30)).max())
    assert bool((e2 <= (1.0 + z.abs()) * b + 2.0 ** -23 * (1.0 + z.abs())).all())
