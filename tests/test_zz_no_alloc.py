"""The allocation-free tensor-core probe (fetidp_tc_selfcheck_static) against the allocating
one (fetidp_tc_selfcheck).  Both run the same seeded inputs through the same kernels, so each
must meet the usual self-check bound (relative error below 1e-4 against FP64 on the same BF16
inputs) and the two must agree.  The file name sorts last, so in a full run it also exercises
the static scratch after every other GPU test of the process."""
import re
from pathlib import Path

import pytest

from paper_2308_11371_gb300 import binding

ROOT = Path(__file__).resolve().parents[1]


@pytest.mark.gpu
@pytest.mark.parametrize("M,K,N", [
    (128, 64, 64),      # one tile of each operand
    (256, 192, 300),    # 64-wide column tiles, ragged columns
    (200, 72, 900),     # ragged rows and K
])
def test_static_probe_matches_allocating_probe(M, K, N):
    import torch
    assert torch.cuda.is_available()
    ref = binding.tc_selfcheck(M, K, N)
    assert ref < 1e-4, ref
    for call in range(2):   # the second call reuses the scratch the first one left behind
        err = binding.tc_selfcheck_static(M, K, N)
        assert err < 1e-4, (call, err)
        assert abs(err - ref) <= 1e-6, (call, err, ref)


@pytest.mark.gpu
def test_static_probe_on_a_side_stream():
    import torch
    ref = binding.tc_selfcheck(256, 192, 300)
    side = torch.cuda.Stream()
    for _ in range(2):
        err = binding.tc_selfcheck_static(256, 192, 300, stream=side.cuda_stream)
        assert abs(err - ref) <= 1e-6, (err, ref)


def test_oversized_probe_is_rejected_before_any_cuda_call():
    """A shape beyond the static scratch fails with EINVAL and names both byte counts; the
    check is host arithmetic, so it also holds on a machine without a GPU."""
    with pytest.raises(binding.FetidpError) as e:
        binding.tc_selfcheck_static(570, 570, 10000)
    assert e.value.status == -1
    msg = str(e.value)
    assert "static scratch holds 4194304" in msg and re.search(r"needs \d+ bytes", msg), msg


def test_header_states_the_scratch_size():
    h = (ROOT / "include" / "fetidp.h").read_text()
    m = re.search(r"#define FETIDP_TC_STATIC_SCRATCH_BYTES (\d+)", h)
    assert m and int(m.group(1)) == binding.TC_STATIC_SCRATCH_BYTES
