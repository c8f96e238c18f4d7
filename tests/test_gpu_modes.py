"""Memory sums in auxiliary-variable form (needs a GPU): for kernels that are
sums of damped modes the recursive sums give the forces of the written-out
convolution -- against the FP64 oracle (which evaluates Eq.
dissipative_force2 term by term from the history), right after they are
built from the ring, after thousands of recursive updates, and with the slow
tail of the suspension; kernels that are not such sums are rejected."""
import numpy as np
import pytest

import oracle
from gld_cases import make_gpu, oracle_from_gpu, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _w(name):
    from paper_1808_00270_gb300 import inputs
    return inputs.WORKLOADS[name]


def _suspension(n=2000, seed=81):
    from paper_1808_00270_gb300 import inputs
    return inputs.Workload("modes_tail", n=n, box=inputs.box_for_density(n, 0.1), m_max=400, dt=0.005, r_c=2.5,
                           tau_s=0.5, tau_p=0.3, steps=1, tail=True, seed=seed)


def _one_step_vs_oracle(w, gpu):
    from paper_1808_00270_gb300 import ARR_DISP, ARR_FC, ARR_FD, ARR_FR
    ref = oracle_from_gpu(w, gpu)
    d0 = gpu.get(ARR_DISP)
    gpu.step(1)
    ref.step(1)
    errs = {"fd": rel_l2(gpu.get(ARR_FD), ref.get(oracle.FD)), "fr": rel_l2(gpu.get(ARR_FR), ref.get(oracle.FR)),
            "fc": rel_l2(gpu.get(ARR_FC), ref.get(oracle.FC)),
            "disp": rel_l2(gpu.get(ARR_DISP) - d0, ref.get(oracle.DISP)),
            "vel": rel_l2(gpu.get_state()[1], ref.get(oracle.VEL))}
    return errs


@pytest.mark.parametrize("warm", [0, 130, 250])
def test_modes_forces_match_oracle(warm):
    """Modes set before the first step, history empty, partial and full:
    one-step F^D, F^R, F^C and displacement within 1e-5 of the oracle."""
    from paper_1808_00270_gb300 import inputs
    w = _w("gld_n4096_m200")
    gpu = make_gpu(w)
    gpu.set_memory_modes(*inputs.memory_modes(w))
    gpu.step(warm)
    errs = _one_step_vs_oracle(w, gpu)
    assert max(errs.values()) < 1e-5, errs


def test_modes_built_from_the_ring_mid_run():
    """Switching from the ring convolution to the modes after 300 steps: the
    sums are rebuilt from the ring and the next step's forces match."""
    from paper_1808_00270_gb300 import inputs
    w = _w("gld_n4096_m200")
    gpu = make_gpu(w)
    gpu.step(300)
    gpu.set_memory_modes(*inputs.memory_modes(w))
    errs = _one_step_vs_oracle(w, gpu)
    assert max(errs.values()) < 1e-5, errs


def test_modes_stay_accurate_over_long_runs_with_the_slow_tail():
    """m_max = 400 with the slow tail (|z| = 0.9975 per step) and r_c = 2.5:
    after 3000 recursive updates (7 passes through the ring) the forces and
    the new velocities still match the written-out convolution."""
    from paper_1808_00270_gb300 import inputs
    w = _suspension()
    gpu = make_gpu(w)
    gpu.set_memory_modes(*inputs.memory_modes(w))
    gpu.step(3000)
    errs = _one_step_vs_oracle(w, gpu)
    print("recursive memory, one-step errors after 3000 steps:", errs)
    # the displacement accumulated over 3000 steps is O(1): one step's share
    # of it carries its FP32 rounding, so the step is judged by V_{n+1}
    errs.pop("disp")
    assert max(errs.values()) < 1e-5, errs


def test_modes_trajectory_matches_ring_path():
    """The recursive path and the ring convolution integrate the same system:
    150 steps from the same state agree to the trajectory tolerance."""
    from paper_1808_00270_gb300 import ARR_DISP, inputs
    w = _w("gld_n4096_m200")
    a, b = make_gpu(w), make_gpu(w)
    b.set_memory_modes(*inputs.memory_modes(w))
    a.step(150)
    b.step(150)
    assert rel_l2(b.get(ARR_DISP), a.get(ARR_DISP)) < 1e-4
    assert rel_l2(b.get_state()[1], a.get_state()[1]) < 1e-3


def test_modes_rejected_when_they_do_not_represent_the_kernels():
    from paper_1808_00270_gb300 import Batch, GLDError, inputs
    from paper_1808_00270_gb300.binding import E_INVAL
    w = _w("gld_n4096_m200")
    g = make_gpu(w)
    rates, omegas = inputs.memory_modes(w)
    for r, o in ((rates[1:], omegas[1:]),                   # the damped cosine left out
                 (rates, omegas * 1.01),                    # wrong frequency
                 (np.append(rates, rates[0]), np.append(omegas, omegas[0])),  # a mode twice
                 (-rates, omegas)):                         # growing modes
        with pytest.raises(GLDError) as e:
            g.set_memory_modes(r, o)
        assert e.value.status == E_INVAL
    g.set_memory_modes(rates, omegas)
    with pytest.raises(GLDError):
        Batch().add(g)
    g.set_memory_modes([], [])  # back to the ring
    Batch().add(g)
