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


@pytest.mark.parametrize("M0,M1,K,N,nops", [
    (120, 8, 120, 4096, 32),    # F_dd stacked with (T_dr U_rp)^T, 32-wide tiles, 2 buffers x 16 ops
    (56, 8, 56, 16, 2),         # tiny ragged case
    (570, 0, 120, 4096, 8),     # U_rd: 5 row tiles, 128-wide column tiles
    (120, 8, 570, 300, 5),      # long K resident in shared memory, ragged columns
    (120, 0, 120, 4096, 32),    # F_dd alone: also the resident-operator kernel (16 groups)
    (56, 0, 56, 16, 3),         # resident-operator kernel, tiny, a one-principal last group
    (100, 0, 64, 1000, 5),      # resident-operator kernel, one k tile, ragged columns
])
def test_tc_combine_matches_fp64_on_bf16_inputs(M0, M1, K, N, nops):
    import torch
    from paper_2308_11371_gb300 import binding
    assert torch.cuda.is_available()
    err = binding.tc_comb_selfcheck(M0, M1, K, N, nops)
    assert err < 1e-4, err
