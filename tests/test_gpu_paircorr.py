"""Distance-binned pair correlations C^a(R,t), C^c(R,t) on the GPU (Sec. III A;
needs a GPU): against their definition on the recorded GPU trajectory (the
pair set and bins replicated in FP32 exactly as the kernels compute them),
against the FP64 oracle from the same initial state, bitwise across graph
forms, and the argument checks."""
import numpy as np
import pytest

import oracle
from gld_cases import make_gpu, make_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _workload(n=500, rho=0.1, m_max=80, seed=71):
    from paper_1808_00270_gb300 import inputs
    return inputs.Workload("pc", n=n, box=inputs.box_for_density(n, rho), m_max=m_max, dt=0.005, r_c=2.0,
                           tau_s=0.5, tau_p=0.3, steps=1, tail=True, seed=seed)


def _pairs_f32(P, box, rmax, nbins):
    """Pairs i < j with r < rmax and their bins, in the kernels' FP32 order:
    d = x_i - x_j, one periodic shift, r2 = (dx dx + dy dy) + dz dz,
    r = sqrt(r2), bin = int(r * float(nbins / rmax))."""
    p = P.astype(np.float32)
    L = np.float32(box)
    half = np.float32(0.5) * L
    n = p.shape[0]
    iu, ju = np.triu_indices(n, 1)
    d = (p[iu] - p[ju]).astype(np.float32)
    d = np.where(d > half, d - L, np.where(d < -half, d + L, d)).astype(np.float32)
    r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    sel = r2 < np.float32(rmax * rmax)
    r = np.sqrt(r2[sel])
    b = np.minimum((r * np.float32(nbins / rmax)).astype(np.int64), nbins - 1)
    e = d[sel].astype(np.float64) / r.astype(np.float64)[:, None]
    return iu[sel], ju[sel], b, e


def _definition(P, V, box, rmax, nbins, L, stride, burn, t_first):
    sa, sc = np.zeros((L, nbins)), np.zeros((L, nbins))
    cnt = np.zeros((L, nbins), dtype=np.int64)
    for t in range(t_first, len(P)):
        i, j, b, e = _pairs_f32(P[t], box, rmax, nbins)
        vit, vjt = (V[t][i] * e).sum(1), (V[t][j] * e).sum(1)
        for t0 in range(burn, t + 1, stride):
            lag = t - t0
            if lag >= L:
                continue
            vi0, vj0 = (V[t0][i] * e).sum(1), (V[t0][j] * e).sum(1)
            np.add.at(sa[lag], b, vit * vi0 + vjt * vj0)
            np.add.at(sc[lag], b, vit * vj0 + vjt * vi0)
            np.add.at(cnt[lag], b, 1)
    safe = np.maximum(cnt, 1)
    return np.where(cnt > 0, sa / (2 * safe), 0.0), np.where(cnt > 0, sc / (2 * safe), 0.0), cnt


def test_pair_correlation_definition():
    """The accumulators equal the definition evaluated on the GPU's own
    recorded positions and velocities (same pairs and bins, FP32 replicated);
    sums to FP32 rounding of the dot products."""
    w = _workload()
    L, stride, burn, nbins = 12, 3, 4, 5
    g = make_gpu(w, vacf_len=L, vacf_stride=stride, vacf_burnin=burn, use_graphs=False)
    g.set_pair_correlation(nbins, w.r_c)
    P, V = [], []
    p, v = g.get_state()
    P.append(p)
    V.append(v)
    for _ in range(1, 50):
        g.step(1)
        p, v = g.get_state()
        P.append(p)
        V.append(v)
    wa, wc, wn = _definition(P, V, w.box, w.r_c, nbins, L, stride, burn, t_first=1)
    ca, cc, cnt = g.pair_correlation()
    assert np.array_equal(cnt, wn) and wn.sum() > 1000
    scale = np.max(np.abs(wa))
    assert np.max(np.abs(ca - wa)) < 1e-5 * scale
    assert np.max(np.abs(cc - wc)) < 1e-5 * scale


def test_pair_correlation_matches_oracle():
    """GPU and FP64 oracle from the same initial state and noise stream, 150
    steps: counts within a few pair samples (bin edges), C^a and C^c within
    1e-3 of the largest |C^a| (trajectories agree to ~1e-5)."""
    w = _workload(n=400, seed=72)
    kw = dict(vacf_len=30, vacf_stride=10, vacf_burnin=20)
    nbins = 4
    g = make_gpu(w, **kw)
    g.set_pair_correlation(nbins, w.r_c)
    ref = make_oracle(w, **kw)
    assert ref.set_paircorr(nbins, w.r_c) == 0
    g.step(150)
    ref.step(150)
    ca, cc, cnt = g.pair_correlation()
    ra, rc, rn = ref.paircorr()
    assert np.max(np.abs(cnt - rn)) <= 3 and rn.sum() > 1000
    scale = np.max(np.abs(ra))
    assert np.max(np.abs(ca - ra)) < 1e-3 * scale
    assert np.max(np.abs(cc - rc)) < 1e-3 * scale


def test_pair_correlation_reproducible_across_graph_forms():
    """Fixed-point per-step sums: graph replay (both forms), eager launches and
    any chunking of the steps give the same bits."""
    w = _workload(n=2000, seed=73)
    kw = dict(vacf_len=40, vacf_stride=8, vacf_burnin=16)
    out = []
    for ug, chunks in ((True, (200,)), (False, (200,)), (2, (64, 7, 129))):
        g = make_gpu(w, use_graphs=ug, **kw)
        g.set_pair_correlation(8, w.r_c)
        for k in chunks:
            g.step(k)
        out.append(g.pair_correlation())
    for o in out[1:]:
        for x, y in zip(out[0], o):
            assert np.array_equal(x, y)


def test_pair_correlation_arguments():
    from paper_1808_00270_gb300 import Batch, GLDError
    from paper_1808_00270_gb300.binding import E_INVAL
    w = _workload(n=300, seed=74)
    g = make_gpu(w)  # no VACF
    with pytest.raises(GLDError) as e:
        g.set_pair_correlation(4, 1.0)
    assert e.value.status == E_INVAL
    h = make_gpu(w, vacf_len=64, vacf_stride=2)
    for nb, rmax in ((0, 1.0), (4, 0.0), (4, w.r_c * 1.01), (100, 1.0)):  # 32 origins x 100 bins > 2048
        with pytest.raises(GLDError):
            h.set_pair_correlation(nb, rmax)
    h.set_pair_correlation(4, 1.5)
    with pytest.raises(GLDError):
        Batch().add(h)  # single contexts only
    h.step(200)  # past the default burn-in of 2 m_max = 160 steps
    ca, cc, cnt = h.pair_correlation()
    assert ca.shape == (64, 4) and cnt.sum() > 0
    h.set_pair_correlation(2, 2.0)  # resetting clears the sums
    ca, cc, cnt = h.pair_correlation()
    assert cnt.sum() == 0 and ca.shape == (64, 2)
