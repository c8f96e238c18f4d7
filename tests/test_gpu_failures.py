"""Failure detection of the GPU path, every failure made on the host (needs a
GPU): a non-finite velocity, a neighbour list pushed past its capacity, and
an allocation refused while new kernels are set.  None of these faults the
device: the non-finite value only travels through arithmetic (every distance
test with it is false), and the list writes are clamped at the capacity.
Each is read back as the documented status code, and the device-side ones
stay latched."""
import numpy as np
import pytest

from gld_cases import make_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _status(fn):
    from paper_1808_00270_gb300 import GLDError
    try:
        fn()
    except GLDError as e:
        return e.status
    return 0


def test_nonfinite_velocity_latches():
    """A NaN in one velocity gives a non-finite displacement at the next step:
    the synchronizing call returns GLD_E_NONFINITE, and so does every later
    call that would launch work (the error is latched)."""
    from paper_1808_00270_gb300 import ARR_VEL, inputs
    from paper_1808_00270_gb300.binding import E_NONFINITE
    w = inputs.MEDIUM
    g = make_gpu(w)
    g.step(3)
    _, v = g.get_state()
    v[17, 1] = np.nan
    g.set(ARR_VEL, v)
    g.step(1)
    assert _status(g.sync) == E_NONFINITE
    assert _status(lambda: g.step(1)) == E_NONFINITE
    assert _status(g.sync) == E_NONFINITE
    g.close()


def test_neighbour_list_overflow_latches():
    """200 particles moved within 0.1 r_c of one point have 199 neighbours
    each, far above the list capacity sized for the creation density: the
    rebuild that follows the new positions reports GLD_E_STATE, and the
    context refuses to step from then on."""
    from paper_1808_00270_gb300 import ARR_POS, inputs
    from paper_1808_00270_gb300.binding import E_STATE
    w = inputs.MEDIUM
    g = make_gpu(w)
    assert g.diag()["maxnb"] < 199
    g.step(2)
    p, _ = g.get_state()
    rng = np.random.default_rng(3)
    p[:200] = 0.5 * w.box + rng.uniform(-0.05 * w.r_c, 0.05 * w.r_c, (200, 3))
    assert _status(lambda: g.set(ARR_POS, p)) == E_STATE
    assert _status(lambda: g.step(1)) == E_STATE
    g.close()


class _RefusingCuda:
    """Stands in for torch.cuda inside the binding's allocator callbacks:
    every allocation is refused, frees pass through."""

    def __init__(self, cuda):
        self._cuda = cuda

    def caching_allocator_alloc(self, *args, **kw):
        raise MemoryError("allocation refused by the test")

    def caching_allocator_delete(self, ptr):
        self._cuda.caching_allocator_delete(ptr)


class _Refusing:
    def __init__(self, torch_mod):
        self.cuda = _RefusingCuda(torch_mod.cuda)


def test_set_kernels_allocation_failure_leaves_no_kernels():
    """A second gld_set_kernels whose table allocation fails returns
    GLD_E_NOMEM; the old tables are already released, so the context must
    then refuse to step (GLD_E_STATE) instead of reading them.  Setting the
    kernels again with the allocator back restores a working context."""
    from paper_1808_00270_gb300 import inputs
    from paper_1808_00270_gb300.binding import E_NOMEM, E_STATE
    from gld_cases import kernels
    w = inputs.MEDIUM
    g = make_gpu(w)
    g.step(5)
    g.sync()
    ks, gk, f, dr = kernels(w)
    real = g._alloc._torch
    g._alloc._torch = _Refusing(torch)
    try:
        assert _status(lambda: g.set_kernels(ks, g=gk, f=f, dr=dr)) == E_NOMEM
    finally:
        g._alloc._torch = real
    assert _status(lambda: g.step(1)) == E_STATE
    g.set_kernels(ks, g=gk, f=f, dr=dr)
    g.step(70)
    g.sync()
    g.close()
