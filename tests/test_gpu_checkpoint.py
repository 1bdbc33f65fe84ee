"""Checkpoint and resume through the C ABI: a run saved at step 30 and resumed in a fresh
batch continues bit for bit like the uninterrupted run (FP32 and FP64, a ragged batch, a
q(t) schedule), and files of another configuration or with a changed byte are refused."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

MEAN = (0.0, 0.0, 1.0, 0.0, 0.0, 0.0)


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2310_03636_gb300 import binding
    return binding


def _fields(b):
    return [p.cpu().clone() for p in b.psi] if not b.uniform else [b.psi.cpu().clone()]


@pytest.mark.parametrize("dtype,shape,ntraj,knots", [
    ("c64", (128, 128), 3, None),
    ("c128", (64, 64, 64), 1, [0.2, 0.05, 0.1]),
    ("c64", [(256,), (64, 64), (8192,)], None, None),
])
def test_resume_is_bitwise(B, tmp_path, dtype, shape, ntraj, knots):
    kw = dict(dtype=dtype, c0=1.0, c1=-0.1, q=0.09, dt=0.02)
    if knots is not None:
        kw.update(q_knots=knots, t_end=60 * 0.02)
    make = (lambda: B.GPEBatch(shape, ntraj, **kw)) if ntraj else (lambda: B.GPEBatch(list(shape), **kw))
    path = tmp_path / "run.ckpt"
    a = make()
    a.init_noise(17, MEAN, 0.5)
    a.step(30)
    a.save(path)
    a.step(20)
    assert a.sync_status() == B.GPE_OK
    ref = _fields(a)
    a.close()
    b = make()              # fresh batch: zero fields, step 0
    b.load(path)
    assert b.step_count == 30
    b.step(20)
    assert b.sync_status() == B.GPE_OK
    for x, y in zip(ref, _fields(b)):
        assert torch.equal(x, y)
    b.close()


def test_refuses_other_configurations_and_corrupt_files(B, tmp_path):
    path = tmp_path / "run.ckpt"
    a = B.GPEBatch((64, 64), 2, "c64", dt=0.02)
    a.init_noise(3, MEAN, 0.5)
    a.save(path)
    for other in (B.GPEBatch((64, 64), 2, "c64", dt=0.01), B.GPEBatch((64, 64), 2, "c128", dt=0.02),
                  B.GPEBatch((64, 64), 3, "c64", dt=0.02), B.GPEBatch((64, 128), 2, "c64", dt=0.02)):
        with pytest.raises(B.GPEError) as ei:
            other.load(path)
        assert ei.value.status == B.GPE_EINVAL
        other.close()
    raw = bytearray(path.read_bytes())
    raw[len(raw) // 2] ^= 1
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(bytes(raw))
    with pytest.raises(B.GPEError) as ei:
        a.load(bad)
    assert "corrupt" in str(ei.value)
    with pytest.raises(B.GPEError):
        a.load(tmp_path / "missing.ckpt")
    (tmp_path / "short.ckpt").write_bytes(bytes(raw[:100]))
    with pytest.raises(B.GPEError):
        a.load(tmp_path / "short.ckpt")
    a.load(path)
    assert a.sync_status() == B.GPE_OK
    a.close()
