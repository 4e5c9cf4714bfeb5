"""The bandwidth probes that supply the roofline denominators do the work they claim."""
import pytest
import torch

from gpu_util import ensure_lib
from paper_2601_10819_gb300 import msda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return ensure_lib()


@pytest.mark.parametrize("blocks,reps,rows", [(1, 1, 3), (4, 2, 16)])
def test_reduce_probe_adds_one_per_row_element(blocks, reps, rows):
    buf = torch.zeros(64 * 256, device="cuda")  # 64 rows of 1 KB
    msda.probe_reduce(buf, reps, blocks, rows)
    torch.cuda.synchronize()
    # every warp (16 per 512-thread block) adds 1.0 to all 256 floats of `rows` rows per rep
    assert float(buf.sum()) == blocks * 16 * reps * rows * 256
    assert torch.all(buf == buf.round()) and float(buf.min()) >= 0


def test_read_probes_run_and_leave_the_buffer_alone():
    buf = torch.randint(0, 255, (1 << 20,), dtype=torch.uint8, device="cuda")
    ref = buf.clone()
    msda.probe_read(buf, 2, 8)            # streaming
    msda.probe_read(buf, 2, 8, rows=16)   # random 512-byte rows
    torch.cuda.synchronize()
    assert torch.equal(buf, ref)
    assert msda.device_status() == 0
