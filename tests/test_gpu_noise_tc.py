"""The colored-noise filter on the tensor cores (needs a GPU): F^R of Eq.
noise_production against the FP64 oracle's direct sum for windows that start
at offsets spread over the filter's 64-row accumulation groups (including
blocks that start before the memory window is filled, n0 < m_max - 1), for stream counts that leave a
partial last tile, and for memory lengths from 32 to 1000; and F^R of a given
time does not depend on where its 64-step block started (the result of a
checkpointed run does not depend on where it was resumed)."""
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


def _w(n, m_max, rho=0.1, seed=7):
    """Short memories take the 64-particle workload's time scales (dt = 0.01,
    tau_s = 0.2): with dt = 0.005 and tau_s = 0.5 a window of 32 steps cuts
    the kernel too sharply to be positive definite."""
    from paper_1808_00270_gb300 import inputs
    short = m_max < 58
    return inputs.Workload(f"tc_n{n}_m{m_max}", n=n, box=inputs.box_for_density(n, rho), m_max=m_max,
                           dt=0.01 if short else 0.005, r_c=2.0, tau_s=0.2 if short else 0.5,
                           tau_p=0.1 if short else 0.3, steps=1, tail=not short, seed=seed)


@pytest.mark.parametrize("n,m_max,rho", [(1500, 400, 0.2), (77, 32, 0.1), (4096, 200, 0.1), (500, 1000, 0.1)])
def test_filter_matches_oracle_at_window_offsets(n, m_max, rho):
    """One step's F^R within 1e-5 of the oracle after set_step to steps whose
    window start n0 - (m_max - 1) falls at different offsets of a 64-row group."""
    from paper_1808_00270_gb300 import ARR_FR
    w = _w(n, m_max, rho)
    g = make_gpu(w)
    for n0 in (0, 5, 17, 64, 93, 1234):
        g.set_step(n0)
        ref = oracle_from_gpu(w, g)
        g.step(1)
        ref.step(1)
        err = rel_l2(g.get(ARR_FR), ref.get(oracle.FR))
        assert err < 1e-5, (n0, err)
    g.close()


def test_filter_result_independent_of_block_start():
    """F^R depends only on the counter-based white noise and the taps, so the
    row of time 200 is the same bits whether its block started at 200, at
    180 or at 137."""
    from paper_1808_00270_gb300 import ARR_FR
    w = _w(1500, 400, 0.2)
    rows = []
    for start in (200, 180, 137):
        g = make_gpu(w)
        g.set_step(start)
        g.step(200 - start + 1)
        assert g.step_index == 201
        rows.append(g.get(ARR_FR))
        g.close()
    assert np.array_equal(rows[0], rows[1]) and np.array_equal(rows[0], rows[2])
