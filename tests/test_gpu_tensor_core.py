"""tcgen05 BF16 GEMM (TMEM accumulator, bulk-copy ring) against an FP64 GEMM of the same
BF16-rounded inputs.  Products of BF16 numbers are exact in FP32, so the only difference is
FP32 accumulation order: a relative error below 1e-4 at K <= 2048 means the layout, swizzle,
descriptors and epilogue are right (a wrong layout gives O(1) errors)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,K,N", [
    (128, 64, 64),        # one tile of each operand
    (256, 192, 300),      # 64-wide column tiles, ragged columns
    (570, 570, 10000),    # 128-wide column tiles, ragged rows and K
    (120, 2048, 40000),   # 256-wide column tiles, long K
])
def test_tc_gemm_matches_fp64_on_bf16_inputs(M, K, N):
    import torch
    from paper_2308_11371_gb300 import binding
    assert torch.cuda.is_available()
    err = binding.tc_selfcheck(M, K, N)
    assert err < 1e-4, err
