"""Checkpoint and restart (cmrt_save / cmrt_load): a run restarted from a
checkpoint continues bit for bit, in FP32 and in 16-bit storage, from host
or device memory and into a fresh context; a checkpoint of another lattice
or a short buffer is refused without touching the state."""
import numpy as np
import pytest

from paper_2005_04642_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2005_04642_gb300 import cmrt as cm  # noqa: E402

cm.load()


def _drop(precision, wall=False):
    d, rn, u = I.static_drop(n=40, radius=10.0)
    return dict(d, precision=precision, wall_y=wall), rn, u


@pytest.mark.parametrize("precision,wall", [(0, False), (0, True), (2, False), (1, True)])
def test_restart_continues_bit_for_bit(precision, wall):
    d, rn, u = _drop(precision, wall)
    a = cm.Lattice(d, rn, u)
    a.step(7)
    ck = a.save()
    a.step(41)  # an odd count past the 32-step graphs: graph replay and single launches
    ref, t_ref = a.populations(), a.time
    a.load(ck)  # host checkpoint
    assert a.time == 7
    a.step(41)
    assert a.time == t_ref
    assert torch.equal(a.populations(), ref)
    # a fresh context of the same lattice, from a device copy of the checkpoint
    b = cm.Lattice(d, None, None)
    b.load(torch.from_numpy(ck).cuda())
    assert b.time == 7
    b.step(41)
    assert torch.equal(b.populations(), ref)
    a.close()
    b.close()


def test_mismatched_or_short_checkpoints_are_refused():
    d, rn, u = _drop(0)
    a = cm.Lattice(d, rn, u)
    a.step(3)
    ck = a.save()
    before = a.populations()
    other = cm.Lattice(dict(d, nx=48), None, None)
    with pytest.raises(cm.CmrtError) as ei:
        other.load(ck)
    assert ei.value.status == cm.CMRT_EINVAL
    f16 = cm.Lattice(dict(d, precision=2), rn, u)
    with pytest.raises(cm.CmrtError) as ei:
        f16.load(ck)
    assert ei.value.status == cm.CMRT_EINVAL
    with pytest.raises(cm.CmrtError) as ei:
        a.load(ck[:-4])
    assert ei.value.status == cm.CMRT_EINVAL
    bad = ck.copy()
    bad[:8] = 0  # not a checkpoint
    with pytest.raises(cm.CmrtError) as ei:
        a.load(bad)
    assert ei.value.status == cm.CMRT_EINVAL
    # refusals leave the state and the context usable
    assert torch.equal(a.populations(), before) and a.time == 3
    a.step(1)
    for lat in (a, other, f16):
        lat.close()
