"""The allocation-free neighbour search (gld_pairs_noalloc) returns the same
pairs as the context-based gld_get_pairs and as the oracle's FP32 brute force
(same FP32 positions, the single-precision distance test of gld.h), on two
calls in a row, for ragged sizes and with particles on the periodic faces.
It exists for callers that cannot allocate device memory; its scratch is a
static device array shared by every call.  Collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _reference_pairs(pos, box, rc):
    from paper_1808_00270_gb300 import GLD
    g = GLD(n=len(pos), box=box, dt=0.01, m_max=4, r_c=rc, pos=pos, vel=np.zeros_like(pos))
    p32, _ = g.get_state()
    want = {tuple(x) for x in g.pairs().tolist()}
    g.close()
    return p32, want


def _positions(n, box, faces, seed):
    """Uniform FP32 positions in [0, box); with `faces`, a quarter of the
    particles get one coordinate on a periodic face (0 or the largest FP32
    value below box)."""
    rng = np.random.default_rng(seed)
    p = rng.uniform(0, box, (n, 3)).astype(np.float32)
    if faces:
        top = np.nextafter(np.float32(box), np.float32(0))
        k = np.arange(0, n, 4)
        p[k, rng.integers(0, 3, k.size)] = np.where(rng.random(k.size) < 0.5, np.float32(0), top)
    return p.astype(np.float64)


@pytest.mark.parametrize("n,box,rc,faces", [(4096, 34.47, 2.0, False), (64, 8.0, 2.0, False),
                                            (20000, 60.0, 2.5, False), (77, 9.0, 2.0, True),
                                            (20001, 60.0, 2.5, True)])
def test_noalloc_pairs_match_context_pairs(n, box, rc, faces):
    import oracle
    from paper_1808_00270_gb300.binding import pairs_noalloc
    p32, want = _reference_pairs(_positions(n, box, faces, n), box, rc)
    brute = oracle.pairs_brute_f32(p32.astype(np.float32), box, np.float32(rc * rc))
    assert {(min(a, b), max(a, b)) for a, b in brute.tolist()} == want
    pos4 = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    pos4[:, :3] = torch.from_numpy(p32.astype(np.float32)).cuda()
    cap = 16 * n
    for _ in range(2):  # the static scratch keeps the previous call's contents
        pairs = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        pairs_noalloc(pos4, box, rc, pairs, count)
        torch.cuda.synchronize()
        k = int(count.item())
        assert k == len(want) and k <= cap
        got = {tuple(x) for x in pairs[:k].cpu().numpy().tolist()}
        assert got == want


def test_noalloc_rejects_oversized_input():
    from paper_1808_00270_gb300.binding import NOALLOC_MAX_N, GLDError, pairs_noalloc
    from paper_1808_00270_gb300.binding import E_INVAL
    n = NOALLOC_MAX_N + 1
    pos4 = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    pairs = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(GLDError) as e:
        pairs_noalloc(pos4, 100.0, 2.0, pairs, count)
    assert e.value.status == E_INVAL
