"""The random-access calibration (gde_probe_random_access) through the C ABI: every access
lands inside the buffer and is counted once (the FP32 adds sum to the number of accesses),
and bad arguments are rejected before anything is launched."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gde():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2410_21634_gb300 as m
    m.load()
    return m


@pytest.mark.parametrize("mode", ["load_atomic", "atomic", "red"])
def test_every_access_counted(gde, mode):
    import torch
    buf = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    nops, reps = 1 << 20, 3
    ms = gde.probe_random_access(buf, nops, mode, grid=152 * 4, reps=reps)
    assert ms > 0
    f = buf.view(torch.float32)
    # the adds go to the upper FP32 half of 8-byte words; each word stays far below 2^24
    assert float(f[1::2].double().sum()) == (reps + 1) * nops
    assert float(f[0::2].double().abs().sum()) == 0.0


@pytest.mark.parametrize("mode", ["atomic64", "red64"])
def test_every_64bit_add_counted(gde, mode):
    import torch
    buf = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    nops, reps = 1 << 20, 2
    assert gde.probe_random_access(buf, nops, mode, grid=152 * 4, reps=reps) > 0
    q = buf.view(torch.int64)
    assert int(q.sum()) == (reps + 1) * nops
    assert int(q.view(-1, 4)[:, 1:].abs().sum()) == 0  # only the first word of a sector


def test_loads_leave_buffer_zero(gde):
    import torch
    buf = torch.full((8 << 20,), 7, dtype=torch.uint8, device="cuda")
    assert gde.probe_random_access(buf, 1 << 18, "load", grid=152, reps=1) > 0
    assert int(buf.count_nonzero()) == 0  # zeroed by the call, only read afterwards


def test_fetch_granularity_limit_accepted(gde):
    import torch
    buf = torch.empty(8 << 20, dtype=torch.uint8, device="cuda")
    for lim in (32, 64, 128):
        assert gde.probe_random_access(buf, 1 << 16, "load", grid=152, reps=1, l2_fetch_bytes=lim) > 0


def test_bad_arguments(gde):
    import torch
    buf = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    for kw in (dict(mode=6), dict(mode=-1), dict(grid=0), dict(reps=0), dict(l2_fetch_bytes=48), dict(nops=0)):
        args = dict(nops=1024, mode="load", grid=8, reps=1, l2_fetch_bytes=0)
        args.update(kw)
        with pytest.raises(gde.GdeError) as e:
            gde.probe_random_access(buf, **args)
        assert e.value.status == gde.EINVAL
    with pytest.raises(gde.GdeError) as e:  # not 256-byte aligned
        gde.probe_random_access(buf[16:], 1024, "load", grid=8, reps=1)
    assert e.value.status == gde.EINVAL
