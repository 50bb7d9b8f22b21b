"""Checkpoint / resume through tdse_save_state and tdse_load_state: a run saved
half way and resumed in a new context continues bitwise identically (state, flux
integral, observation history), and the adjoint still works after the resume."""
import numpy as np
import pytest

from paper_2401_07416_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_07416_gb300 import build
    build.build()
    from paper_2401_07416_gb300 import tdse
    return tdse


@pytest.mark.parametrize("precision", ["FP64", "FP32_KAHAN", "FP32"])
def test_save_load_resume_is_bitwise(T, tmp_path, precision):
    from paper_2401_07416_gb300.sim import Sim
    prec = getattr(T, precision)
    g = W.small_grid(40, 28, 48, h=(0.2, 0.2, 0.2), dt=0.004, bc=(0, 0, 1), mask=6,
                     det_k=14, eta=0.3)
    atoms = np.array([[3.9, 2.7, 3.5, 6.0], [1.1, 0.5, 3.2, 8.0]])
    p = W.Packet((4.0, 2.8, 6.5), (0.0, 0.0, 0.8), (0.0, 0.0, -2.0))
    path = str(tmp_path / "run.tdse")
    with Sim(g, precision=prec, ckpt_every=10) as a:
        a.set_atoms(0, atoms)
        a.set_packet(0, p)
        a.step(30)
        a.save(path)
        a.step(25)
        Ra, Ia = a.state(0)
        Fa, ha = a.flux_map(0), a.history(0)
        ga = np.zeros((g.nz, g.ny, g.nx))
        T.tdse_adjoint(a.ctx, 0, 2 * Fa, ga, None)
    with Sim(g, precision=prec, ckpt_every=10) as b:
        b.load(path)
        b.step(25)
        Rb, Ib = b.state(0)
        Fb, hb = b.flux_map(0), b.history(0)
        gb = np.zeros((g.nz, g.ny, g.nx))
        T.tdse_adjoint(b.ctx, 0, 2 * Fb, gb, None)
    assert np.array_equal(Ra, Rb) and np.array_equal(Ia, Ib)
    assert np.array_equal(Fa, Fb)
    assert np.array_equal(ha, hb)
    assert np.array_equal(ga, gb)


def test_load_rejects_other_grid(T, tmp_path):
    from paper_2401_07416_gb300.sim import Sim
    g = W.small_grid(16, 16, 16, h=(0.2, 0.2, 0.2), dt=0.004, bc=(0, 0, 1))
    path = str(tmp_path / "a.tdse")
    with Sim(g, precision=T.FP64) as a:
        a.set_packet(0, W.Packet((1.6, 1.6, 1.6), (0.5, 0.5, 0.5), (0, 0, 1)))
        a.save(path)
    g2 = W.small_grid(20, 16, 16, h=(0.2, 0.2, 0.2), dt=0.004, bc=(0, 0, 1))
    with Sim(g2, precision=T.FP64) as b:
        with pytest.raises(T.TdseError) as e:
            b.load(path)
        assert e.value.status == T.EINVAL
