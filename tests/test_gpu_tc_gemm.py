"""The tcgen05 BF16 GEMM of the surrogate network against float64 products of the same
BF16 values: FP32 accumulation over K terms, so the bound is K x 2^-24 of sum |a||b| (plus
the FP32 rounding of the result)."""
import numpy as np
import pytest

from paper_2109_04469_gb300 import pic

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_04469_gb300 import build as B

    B.build()
    assert torch.cuda.is_available()


# shapes of the network's products (forward at batch 1024, weight gradients with K = batch),
# K tails shorter than a 64-wide stage, N tails shorter than a column tile, N above 256 (several
# column tiles), and more K-stages than the ring holds
@pytest.mark.parametrize("m,n,k", [(128, 16, 16), (128, 256, 256), (256, 192, 256),
                                   (256, 256, 16), (384, 48, 80), (128, 128, 1024),
                                   (1024, 256, 256), (1024, 192, 256), (1024, 256, 16),
                                   (256, 16, 1024), (256, 192, 1024), (128, 208, 64),
                                   (256, 640, 144), (128, 32, 2048)])
def test_gemm_matches_float64(m, n, k):
    g = torch.Generator().manual_seed(m * 7 + n * 3 + k)
    a = torch.randn(m, k, generator=g).to(torch.bfloat16)
    b = torch.randn(n, k, generator=g).to(torch.bfloat16)
    c = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
    pic.tc_gemm_bf16(a.cuda(), b.cuda(), c)
    a64, b64 = a.double().numpy(), b.double().numpy()
    ref = a64 @ b64.T
    bound = np.abs(a64) @ np.abs(b64).T * (k * 2.0**-24) + np.abs(ref) * 2.0**-23 + 1e-30
    err = np.abs(c.cpu().double().numpy() - ref)
    assert np.all(err <= bound), float((err / bound).max())


def test_bad_shapes_are_rejected():
    a = torch.zeros(100, 16, dtype=torch.bfloat16, device="cuda")
    b = torch.zeros(16, 16, dtype=torch.bfloat16, device="cuda")
    c = torch.zeros(100, 16, dtype=torch.float32, device="cuda")
    with pytest.raises(pic.PicError):  # m not a multiple of 128
        pic.tc_gemm_bf16(a, b, c)


def test_misaligned_operand_is_rejected():
    """The TMA tensor maps need 16-byte aligned operands: an offset view is refused on the
    host, before any launch, and c is left untouched."""
    base = torch.zeros(128 * 16 + 1, dtype=torch.bfloat16, device="cuda")
    a = base[1:].view(128, 16)  # 2 bytes past a 256-byte boundary
    b = torch.zeros(16, 16, dtype=torch.bfloat16, device="cuda")
    c = torch.full((128, 16), 7.0, dtype=torch.float32, device="cuda")
    with pytest.raises(pic.PicError) as e:
        pic.tc_gemm_bf16(a, b, c)
    assert e.value.code == -1
    assert bool(torch.all(c == 7.0))
