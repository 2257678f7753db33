"""The tcgen05 BF16 contraction (jagp_gemm_bf16x) against a plain PyTorch
fp32/fp64 reference of the same operation."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SIX = [(0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def split3(torch, x, Kp):
    """FP32 rows -> three BF16 terms side by side, zero-padded to Kp each."""
    M, K = x.shape
    out = torch.zeros((M, 3 * Kp), dtype=torch.bfloat16, device=x.device)
    r = x.float()
    for t in range(3):
        b = r.to(torch.bfloat16)
        out[:, t * Kp:t * Kp + K] = b
        r = r - b.float()
    return out


def reference(torch, A, B, Kp, pairs):
    C = 0
    for a, b in pairs:
        C = C + A[:, a * Kp:(a + 1) * Kp].double() @ B[:, b * Kp:(b + 1) * Kp].double().T
    return C


def scale(torch, A, B, Kp, pairs):
    S = 0
    for a, b in pairs:
        S = S + A[:, a * Kp:(a + 1) * Kp].double().abs() @ B[:, b * Kp:(b + 1) * Kp].double().abs().T
    return S


@pytest.mark.parametrize("M,N,K,pairs", [(300, 320, 320, SIX), (1000, 24, 24, [(0, 0)]),
                                         (256, 1536, 128, [(0, 0), (1, 0)]), (129, 40, 100, SIX)])
def test_umma_matches_reference(torch_cuda, M, N, K, pairs):
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    g = torch.Generator(device="cuda").manual_seed(M + N)
    Kp = (K + 63) // 64 * 64
    x = torch.randn((M, K), device="cuda", generator=g)
    y = torch.randn((N, K), device="cuda", generator=g)
    A, B = split3(torch, x, Kp), split3(torch, y, Kp)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    err = pg.jagp_gemm_bf16x(A, 3, B, 3, Kp, pairs, C)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = reference(torch, A, B, Kp, pairs)
    S = scale(torch, A, B, Kp, pairs)
    d = (C.double() - ref).abs()
    # FP32 accumulation of exact BF16 products
    assert torch.all(d <= 4e-6 * S + 1e-30), float((d / S).max())
    if pairs == SIX:
        # the six-term split reproduces the FP32 operands' product to ~FP32 accuracy
        full = x.double() @ y.double().T
        Sf = x.double().abs() @ y.double().abs().T
        assert torch.all((C.double() - full).abs() <= 4e-6 * Sf), float(((C.double() - full).abs() / Sf).max())


def test_umma_gather_scatter_and_live_count(torch_cuda):
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    M, N, K = 500, 160, 192
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.randn((M, K), device="cuda", generator=g)
    y = torch.randn((N, K), device="cuda", generator=g)
    A, B = split3(torch, x, K), split3(torch, y, K)
    rows = torch.randperm(2 * M, generator=torch.Generator().manual_seed(1))[:M].to(torch.int32).cuda()
    live = 317
    count = torch.tensor([live], dtype=torch.int32, device="cuda")
    out = torch.zeros((2 * M, N), dtype=torch.float32, device="cuda")
    err = pg.jagp_gemm_bf16x(A, 3, B, 3, K, SIX, out, rows=rows, count=count)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = reference(torch, A, B, K, SIX)
    S = scale(torch, A, B, K, SIX)
    r = rows.long()
    assert torch.all((out[r[:live]].double() - ref[:live]).abs() <= 4e-6 * S[:live])
    untouched = torch.ones(2 * M, dtype=torch.bool, device="cuda")
    untouched[r[:live]] = False
    assert torch.all(out[untouched] == 0)


def test_umma_rejects_bad_shapes(torch_cuda):
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    A = torch.zeros((8, 96), dtype=torch.bfloat16, device="cuda")
    C = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(pg.JagpError):
        pg.jagp_gemm_bf16x(A, 1, A, 1, 96, [(0, 0)], C)        # Kp not a multiple of 64
    A = torch.zeros((8, 64), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(pg.JagpError):
        pg.jagp_gemm_bf16x(A, 1, A, 1, 64, [(1, 0)], C)        # term index out of range


def slice_fixed4(torch, x, Kp, nsl=4):
    """Rows -> nsl exact 8-bit slices (as BF16) relative to 2^e, e from the row maximum."""
    M, K = x.shape
    x = x.double()
    _, e = torch.frexp(x.abs().max(dim=1).values)
    e = torch.where(x.abs().max(dim=1).values > 0, e, torch.zeros_like(e))
    xs = x * torch.pow(2.0, (7 - e).double())[:, None]
    out = torch.zeros((M, nsl * Kp), dtype=torch.bfloat16, device=x.device)
    for t in range(nsl):
        q = torch.round(xs)
        out[:, t * Kp:t * Kp + K] = q.to(torch.bfloat16)
        xs = (xs - q) * 256.0
    return out, e.to(torch.int32)


TEN = [(0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0), (0, 3), (1, 2), (2, 1), (3, 0)]
FIFTEEN = TEN + [(0, 4), (1, 3), (2, 2), (3, 1), (4, 0)]
TWENTYONE = FIFTEEN + [(0, 5), (1, 4), (2, 3), (3, 2), (4, 1), (5, 0)]


@pytest.mark.parametrize("M,N,K,nsl", [(300, 320, 320, 4), (129, 24, 24, 4), (200, 1536, 256, 4), (64, 100, 1000, 4),
                                       (300, 320, 320, 5), (129, 200, 4096, 5), (300, 320, 320, 6),
                                       (129, 200, 4096, 6)])
def test_umma_fixed_point_is_exact_up_to_fp32_rounding(torch_cuda, M, N, K, nsl):
    """Exact slice products summed exactly: the result equals the FP64 value
    reconstructed from the same slices to about one FP32 rounding, and the
    slicing itself is within its truncation bound of the FP64 product."""
    torch = torch_cuda
    import paper_2002_07401_gb300 as pg
    g = torch.Generator(device="cuda").manual_seed(M * 7 + K)
    # rows with a wide dynamic range, like orbital values
    x = (torch.randn((M, K), device="cuda", generator=g) *
         torch.exp(-6 * torch.rand((M, K), device="cuda", generator=g))).float()
    y = torch.randn((N, K), device="cuda", dtype=torch.float64, generator=g) * 0.1
    y[:, :min(N, K)] += torch.eye(N, K, device="cuda", dtype=torch.float64)[:, :min(N, K)]
    Kp = (K + 63) // 64 * 64
    pairs = {4: TEN, 5: FIFTEEN, 6: TWENTYONE}[nsl]
    A, ea = slice_fixed4(torch, x, Kp, nsl)
    B, eb = slice_fixed4(torch, y, Kp, nsl)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    err = pg.jagp_gemm_bf16x(A, nsl, B, nsl, Kp, pairs, C, row_exp=ea, col_exp=eb)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    Ad, Bd = A.double(), B.double()
    recon = 0
    for a, b in pairs:
        recon = recon + (Ad[:, a * Kp:(a + 1) * Kp] @ Bd[:, b * Kp:(b + 1) * Kp].T) * 256.0 ** -(a + b)
    scale = torch.pow(2.0, (ea[:, None] + eb[None, :] - 14).double())
    recon = recon * scale
    S = x.double().abs() @ y.abs().T
    d = (C.double() - recon).abs()
    assert torch.all(d <= 3e-7 * recon.abs() + 1e-9 * S), float((d / (recon.abs() + 1e-300)).max())
    # truncation of the slicing: dropped slice pairs and the remainder beyond four slices
    ref = x.double() @ y.T
    bound = K * scale * 2.0 ** 14 * 4 * 256.0 ** -(nsl - 0.5)
    assert torch.all((recon - ref).abs() <= bound)
