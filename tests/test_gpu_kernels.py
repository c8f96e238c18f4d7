"""Kernel-level parity of the CUDA path with the oracle (needs a GPU)."""
import numpy as np
import pytest

import oracle
from gld_cases import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_philox_bit_exact():
    """The GPU's Philox4x32-10 words equal the oracle's, bit for bit, including
    the published known-answer counters."""
    from paper_1808_00270_gb300 import philox_dev
    rng = np.random.default_rng(1)
    keys = [(0, 0), (0xFFFFFFFF, 0xFFFFFFFF), (0xA4093822, 0x299F31D0), (12345, 678)]
    ctr = rng.integers(0, 2 ** 32, size=(4099, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    ctr[2] = [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]
    for key in keys:
        d_ctr = torch.from_numpy(ctr.view(np.int32).copy()).cuda()
        d_out = torch.zeros_like(d_ctr)
        philox_dev(d_ctr, key, d_out)
        torch.cuda.synchronize()
        got = d_out.cpu().numpy().view(np.uint32)
        want = np.array([oracle.philox4x32_10(c, key) for c in ctr])
        assert np.array_equal(got, want), f"philox mismatch for key {key}"


def test_gauss3_matches_oracle():
    """Gaussian components agree with the FP64 oracle to FP32 rounding of
    log / sincos (the uniforms themselves are exact)."""
    from paper_1808_00270_gb300 import gauss3_dev
    rng = np.random.default_rng(2)
    n = 5000
    part = rng.integers(0, 300000, n).astype(np.int32)
    time = rng.integers(-500, 10 ** 6, n).astype(np.int64)
    time[:10] = [-399, -1, 0, 1, 2 ** 40, -(2 ** 40), 7, 8, 9, 10]
    seed = 0x1234_5678_9ABC
    out = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    gauss3_dev(seed, torch.from_numpy(part).cuda(), torch.from_numpy(time).cuda(), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    want = np.array([oracle.gauss3(seed, int(p), int(t)) for p, t in zip(part, time)])
    err = np.abs(got - want) / np.maximum(1.0, np.abs(want))
    assert err.max() < 2e-6, err.max()


def _ring_case(n, m_max, nacc, step, bf16, rng):
    n_pad = (n + 31) // 32 * 32
    H = m_max - 1
    ring = np.zeros((H, 3, n_pad), dtype=np.float32)
    ring[:, :, :n] = rng.normal(0, 0.01, size=(H, 3, n)).astype(np.float32)
    if bf16:
        t = torch.from_numpy(ring).to(torch.bfloat16)
        ring = t.float().numpy()  # the values the kernel will see
        d_ring = t.cuda()
    else:
        d_ring = torch.from_numpy(ring).cuda()
    coef = rng.normal(0, 1, size=(nacc, m_max)).astype(np.float32)
    # hist[m-1] = dR_{step-m} lives at slot (step-m) mod H
    hist = np.stack([ring[(step - m) % H].T[:n] for m in range(1, m_max)])  # [H, n, 3]
    want = oracle.history_projections(hist, coef.astype(np.float64))
    out = torch.zeros((nacc, 3, n_pad), dtype=torch.float32, device="cuda")
    return d_ring, torch.from_numpy(coef).cuda(), out, want, n_pad


@pytest.mark.parametrize("n,m_max,nacc,step", [(1000, 37, 2, 0), (1000, 37, 2, 123), (1100, 64, 3, 5),
                                               (333, 9, 9, 1000001), (4096, 200, 2, 777), (70, 2, 1, 3),
                                               (20000, 400, 2, 12345), (20000, 400, 1, 3), (7000, 130, 3, 64)])
@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("kahan", [False, True])
def test_hist_conv_parity(n, m_max, nacc, step, bf16, kahan):
    """out[a,c,i] = sum_m coef[a,m] dR_{i,c,step-m} on identical inputs, several
    tiles with a ragged tail, coefficient rotation at any step."""
    from paper_1808_00270_gb300 import hist_conv_dev
    rng = np.random.default_rng(n + m_max + nacc)
    d_ring, d_coef, out, want, n_pad = _ring_case(n, m_max, nacc, step, bf16, rng)
    hist_conv_dev(d_ring, n_pad, m_max, step, d_coef, nacc, out, bf16=bf16, kahan=kahan)
    torch.cuda.synchronize()
    got = out.cpu().numpy()[:, :, :n].transpose(0, 2, 1)
    assert rel_l2(got, want) < 1e-5
    assert np.all(out.cpu().numpy()[:, :, n:] == 0)


def test_hist_conv_kahan_reduces_error():
    """Compensated summation over m is closer to the FP64 sum than plain FP32
    accumulation on a long memory with a large mean."""
    from paper_1808_00270_gb300 import hist_conv_dev
    rng = np.random.default_rng(5)
    n, m_max = 2048, 4000
    n_pad = n
    ring = (1.0 + rng.normal(0, 1e-3, size=(m_max - 1, 3, n))).astype(np.float32)
    coef = np.ones((1, m_max), dtype=np.float32) * np.float32(0.1)
    d_ring, d_coef = torch.from_numpy(ring).cuda(), torch.from_numpy(coef).cuda()
    hist = np.stack([ring[(0 - m) % (m_max - 1)].T for m in range(1, m_max)])
    want = oracle.history_projections(hist, coef.astype(np.float64))
    errs = {}
    for kahan in (False, True):
        out = torch.zeros((1, 3, n_pad), dtype=torch.float32, device="cuda")
        hist_conv_dev(d_ring, n_pad, m_max, 0, d_coef, 1, out, kahan=kahan)
        torch.cuda.synchronize()
        errs[kahan] = rel_l2(out.cpu().numpy().transpose(0, 2, 1), want)
    assert errs[True] < 0.1 * errs[False] and errs[True] < 1e-7, errs


@pytest.mark.parametrize("wname", ["gld_n64_m32", "gld_n4096_m200", "gld_n262144_m400"])
def test_noise_coefficients_match_oracle(wname):
    """A_s, K_m, a and b derived on the GPU in FP64 equal the oracle's."""
    from paper_1808_00270_gb300 import inputs
    from gld_cases import make_gpu, make_oracle
    w = inputs.WORKLOADS[wname]
    if w.n > 5000:  # only the kernel tables matter here
        w = inputs.Workload(w.name, n=64, box=w.box, m_max=w.m_max, dt=w.dt, r_c=w.r_c, tau_s=w.tau_s,
                            tau_p=w.tau_p, steps=1, tail=w.tail)
    gpu = make_gpu(w)
    ref = make_oracle(w).coefs()
    c = gpu.coefs()
    assert np.allclose(c["Kd"], ref["Kd"], rtol=1e-13, atol=1e-15)
    assert np.max(np.abs(c["A"] - ref["A"])) < 1e-12 * np.abs(ref["A"]).max()
    assert abs(c["a"] - ref["a"]) < 1e-14 and abs(c["b"] - ref["b"]) < 1e-14
    assert c["spec_min"] > 0


def test_not_psd_is_rejected():
    from paper_1808_00270_gb300 import GLD, GLDError
    from paper_1808_00270_gb300.binding import E_NOT_PSD
    M = 8
    Kd = np.zeros(M)
    Kd[0], Kd[1] = 0.05, 0.5
    rng = np.random.default_rng(0)
    g = GLD(n=16, box=10.0, dt=0.1, m_max=M, r_c=2.0, pos=rng.uniform(0, 10, (16, 3)),
            vel=np.zeros((16, 3)))
    with pytest.raises(GLDError) as e:
        g.set_kernels(Kd, discrete=True)
    assert e.value.status == E_NOT_PSD
    g2 = GLD(n=16, box=10.0, dt=0.1, m_max=M, r_c=2.0, pos=rng.uniform(0, 10, (16, 3)),
             vel=np.zeros((16, 3)), psd_clamp=True)
    g2.set_kernels(Kd, discrete=True)
    assert g2.coefs()["clamped_mass"] > 0


def _pairs_gpu_vs_oracle(pos, box, rc):
    from paper_1808_00270_gb300 import GLD
    n = len(pos)
    g = GLD(n=n, box=box, dt=0.01, m_max=4, r_c=rc, pos=pos, vel=np.zeros((n, 3)))
    p32, _ = g.get_state()
    got = {tuple(x) for x in g.pairs().tolist()}
    want = {tuple(x) for x in oracle.pairs_brute_f32(p32.astype(np.float32), box, np.float32(rc * rc)).tolist()}
    return got, want


@pytest.mark.parametrize("n,box,rc", [(64, 8.0, 2.0), (4096, 34.47, 2.0), (20000, 60.0, 2.5), (1, 8.0, 2.0),
                                      (2, 8.0, 3.9), (500, 7.0, 3.5), (3000, 20.0, 1.0)])
def test_neighbor_pairs_bit_exact(n, box, rc):
    """The cell-list traversal finds exactly the pairs of the brute-force FP32
    search on the same positions."""
    rng = np.random.default_rng(n)
    pos = rng.uniform(0, box, (n, 3))
    if n > 10:  # particles on and next to the periodic faces
        pos[: n // 10, 0] = rng.choice([0.0, 1e-7, box - 1e-7, box / 2], n // 10)
    got, want = _pairs_gpu_vs_oracle(pos, box, rc)
    assert got == want
