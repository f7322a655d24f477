"""The read-bandwidth probe behind the roofline's L2 and HBM figures: it
runs, leaves its buffer unchanged, rejects unaligned or ragged buffers on the
host, and reads an L2-resident buffer faster than one far larger than L2."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu(libsoc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rate(ctx, buf, reps):
    s = torch.cuda.current_stream()
    ctx.probe_read(buf, reps, stream=s)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    ctx.probe_read(buf, reps, stream=s)
    b.record(s)
    torch.cuda.synchronize()
    return buf.numel() * buf.element_size() * reps / (a.elapsed_time(b) / 1e3) / 1e9


def test_probe_read(libsoc):
    ctx = libsoc.Context(0, 1)
    buf = torch.arange(1 << 18, dtype=torch.int32, device="cuda")
    ref = buf.clone()
    ctx.probe_read(buf, 3)
    torch.cuda.synchronize()
    assert torch.equal(buf, ref)
    with pytest.raises(Exception):
        ctx.probe_read(buf[1:], 1)          # 4-byte offset: not 16-byte aligned
    with pytest.raises(Exception):
        ctx.probe_read(buf[:5], 1)          # 20 bytes: not a multiple of 16
    with pytest.raises(Exception):
        ctx.probe_read(buf, 0)
    l2 = _rate(ctx, torch.ones(8 << 18, dtype=torch.float32, device="cuda"), 64)        # 8 MiB
    hbm = _rate(ctx, torch.ones(2048 << 18, dtype=torch.float32, device="cuda"), 1)     # 2 GiB
    assert l2 > 1.2 * hbm > 0, (l2, hbm)
    ctx.close()
