"""The serving loop (needs a GPU): admission by device bytes, continuous
batching, and results that do not depend on the other requests."""
import numpy as np
import pytest

from gld_cases import kernels, make_gpu, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _workload(name, n, rho, m_max, seed):
    from paper_1808_00270_gb300 import inputs
    return inputs.Workload(name, n=n, box=inputs.box_for_density(n, rho), m_max=m_max, dt=0.005, r_c=2.0,
                           tau_s=0.5, tau_p=0.3, steps=1, tail=True, seed=seed)


VACF = dict(vacf_len=96, vacf_stride=16, vacf_burnin=64)


def _submit(srv, w, steps, arrival=0.0, keep_state=True):
    from paper_1808_00270_gb300 import inputs
    pos, vel = inputs.initial_state(w)
    ks, g, f, dr = kernels(w)
    return srv.submit(n=w.n, box=w.box, dt=w.dt, m_max=w.m_max, r_c=w.r_c, pos=pos, vel=vel, Ks=ks, g=g, f=f,
                      dr=dr, steps=steps, arrival=arrival, keep_state=keep_state, mass=w.mass, kT=w.kT,
                      A_cons=w.A_cons, seed=w.seed, **VACF)


def _mix():
    return [(_workload("s_n512_m64", 512, 0.05, 64, 21), 640),
            (_workload("s_n3000_m300", 3000, 0.1, 300, 22), 450),   # tail of 2 steps
            (_workload("s_n900_m150", 900, 0.2, 150, 23), 40),      # shorter than one block
            (_workload("s_n200_m80", 200, 0.02, 80, 24), 0),        # no steps
            (_workload("s_n6000_m400", 6000, 0.1, 400, 25), 256)]


TARGET = (_workload("s_n2000_m200", 2000, 0.1, 200, 26), 333)


def test_bytes_needed_is_what_a_context_holds():
    from paper_1808_00270_gb300.binding import bytes_needed
    for w, kw in [(_workload("b1", 1000, 0.1, 100, 1), {}),
                  (_workload("b2", 5000, 0.02, 400, 2), dict(hist_dtype="bf16", vacf_len=200, vacf_stride=10)),
                  (_workload("b3", 333, 0.2, 70, 3), dict(vacf_len=5))]:
        g = make_gpu(w, **kw)
        vk = {k: kw[k] for k in ("vacf_len", "vacf_stride") if k in kw}
        need = bytes_needed(n=w.n, box=w.box, m_max=w.m_max, r_c=w.r_c, dt=w.dt,
                            hist_dtype=kw.get("hist_dtype", "f32"), Q=1, nr=w.nr, **vk)
        assert g.bytes() == need


def test_result_alone_and_in_the_mix_identical():
    """The same request served alone and among others arriving at different
    times returns the same VACF and final state, bit for bit."""
    from paper_1808_00270_gb300 import Server
    a = Server()
    ra = _submit(a, *TARGET)
    a.drain(120)
    alone = a.result(ra)
    assert alone["status"] == 0
    b = Server()
    ids = []
    for k, (w, steps) in enumerate(_mix()):
        ids.append(_submit(b, w, steps, arrival=0.0 if k < 2 else 0.02))
        if k == 1:
            rb = _submit(b, *TARGET, arrival=0.0)
    b.drain(120)
    mixed = b.result(rb)
    assert mixed["status"] == 0
    assert mixed["n_origins"] == alone["n_origins"] > 0
    assert np.array_equal(mixed["vacf"], alone["vacf"])
    assert np.array_equal(mixed["pos"], alone["pos"]) and np.array_equal(mixed["vel"], alone["vel"])
    for i in ids:
        r = b.result(i)
        assert r["status"] == 0 and r["done"] >= r["admitted"] >= r["arrival"]
    st = b.stats()
    assert st["done"] == len(ids) + 1 and st["failed"] == 0 and st["bytes"] == 0


def test_served_request_matches_a_plain_run():
    """A served request integrates the system a plain context integrates (the
    convolution's summation order may differ: FP32 rounding)."""
    from paper_1808_00270_gb300 import ARR_POS, Server
    w, steps = TARGET
    g = make_gpu(w, **VACF)
    g.step(steps)
    c, n = g.vacf()
    p, v = g.get_state()
    s = Server()
    r = _submit(s, w, steps)
    s.drain(120)
    out = s.result(r)
    assert out["n_origins"] == n
    assert np.max(np.abs(out["vacf"] - c)) <= 1e-4 * abs(c[0])
    assert rel_l2(out["vel"], v) < 1e-4
    d = out["pos"] - p
    d -= w.box * np.round(d / w.box)
    assert np.max(np.abs(d)) < 1e-3


def test_admission_respects_the_byte_budget():
    """With a budget for about two systems at a time, no more are resident;
    a request larger than the budget fails alone; the rest complete."""
    from paper_1808_00270_gb300 import Server
    from paper_1808_00270_gb300.binding import E_NOMEM, bytes_needed
    ws = [(_workload("a%d" % k, 1500 + 500 * k, 0.1, 120, 30 + k), 192) for k in range(5)]
    need = [bytes_needed(n=w.n, box=w.box, m_max=w.m_max, r_c=w.r_c, dt=w.dt, Q=1, nr=w.nr, **{
        k: VACF[k] for k in ("vacf_len", "vacf_stride")}) for w, _ in ws]
    budget = need[0] + need[1] + 1  # any three exceed it, each one fits
    assert max(need) <= budget
    s = Server(hbm_budget=budget)
    ids = [_submit(s, w, steps) for w, steps in ws]
    big = _submit(s, _workload("big", 60000, 0.1, 400, 40), 64)
    s.drain(120)
    st = s.stats()
    assert st["bytes_peak"] <= budget and st["members_peak"] <= 2
    assert st["done"] == len(ids) and st["failed"] == 1
    assert s.result(big)["status"] == E_NOMEM
    for i in ids:
        assert s.result(i)["status"] == 0


def test_requests_wait_for_their_arrival():
    from paper_1808_00270_gb300 import Server
    s = Server()
    t0 = s.clock()
    w = _workload("late", 500, 0.1, 64, 50)
    i0 = _submit(s, w, 128, arrival=t0, keep_state=False)
    i1 = _submit(s, w, 128, arrival=t0 + 0.3, keep_state=False)
    s.drain(60)
    r0, r1 = s.result(i0), s.result(i1)
    assert r1["admitted"] >= t0 + 0.3 and r0["done"] > r0["admitted"] >= r0["arrival"]
    assert np.array_equal(r0["vacf"], r1["vacf"])  # same system, same result


def test_cancel_and_forced_drain_timeout():
    """Host-side failure paths: a drain that runs out of time returns
    GLD_E_TIMEOUT and leaves the server usable; a queued and an admitted
    request are cancelled (their memory returns to the budget) while the
    others complete."""
    from paper_1808_00270_gb300 import GLDError, Server
    from paper_1808_00270_gb300.binding import E_CANCELLED, E_TIMEOUT
    s = Server()
    a = _submit(s, _workload("long", 3000, 0.1, 200, 60), 64 * 400, keep_state=False)
    b = _submit(s, _workload("short", 500, 0.1, 64, 61), 256, keep_state=False)
    c = _submit(s, _workload("later", 500, 0.1, 64, 62), 128, arrival=s.clock() + 30.0, keep_state=False)
    with pytest.raises(GLDError) as e:
        s.drain(0.05)
    assert e.value.status == E_TIMEOUT
    assert s.stats()["active"] >= 1
    s.cancel(a)  # admitted
    s.cancel(c)  # still queued
    s.drain(60)
    assert s.result(a)["status"] == E_CANCELLED and s.result(c)["status"] == E_CANCELLED
    assert s.result(b)["status"] == 0
    st = s.stats()
    assert st["bytes"] == 0 and st["failed"] == 2 and st["done"] == 1
    with pytest.raises(GLDError):
        s.cancel(b)  # already finished


def _pn_plain(w, strength, degree):
    from paper_1808_00270_gb300 import GLD, inputs
    from gld_cases import common_kwargs
    pos, vel = inputs.initial_state(w)
    ks, g, f, dr = kernels(w)
    sim = GLD(pos=pos, vel=vel, **common_kwargs(w, **VACF))
    sim.set_kernels(ks, g=g, f=strength * f, dr=dr)
    sim.set_pair_noise(degree)
    return sim


def _pn_submit(srv, w, steps, strength, degree, arrival=0.0):
    from paper_1808_00270_gb300 import inputs
    pos, vel = inputs.initial_state(w)
    ks, g, f, dr = kernels(w)
    return srv.submit(n=w.n, box=w.box, dt=w.dt, m_max=w.m_max, r_c=w.r_c, pos=pos, vel=vel, Ks=ks, g=g,
                      f=strength * f, dr=dr, steps=steps, arrival=arrival, keep_state=True, mass=w.mass, kT=w.kT,
                      A_cons=w.A_cons, r_c_min=w.r_c_min, seed=w.seed, pair_noise=degree, **VACF)


def test_served_pair_noise_matches_a_plain_run():
    """A request with the pair-correlated random force (degree 8, the pair
    kernel at 0.3 of the workload's) integrates what a plain context with
    gld_set_pair_noise(8) integrates, among other requests with and without
    it (FP32 summation orders differ between the batched and the single
    filter: the tolerances of the plain comparison)."""
    from paper_1808_00270_gb300 import Server
    w, steps = TARGET
    sim = _pn_plain(w, 0.3, 8)
    sim.step(steps)
    c, n = sim.vacf()
    p, v = sim.get_state()
    s = Server()
    others = [_submit(s, *_mix()[0]), _pn_submit(s, *_mix()[1], 0.3, 6)]
    r = _pn_submit(s, w, steps, 0.3, 8, arrival=0.01)
    s.drain(120)
    out = s.result(r)
    assert out["status"] == 0 and out["n_origins"] == n
    assert np.max(np.abs(out["vacf"] - c)) <= 1e-4 * abs(c[0])
    assert rel_l2(out["vel"], v) < 1e-4
    d = out["pos"] - p
    d -= w.box * np.round(d / w.box)
    assert np.max(np.abs(d)) < 1e-3
    for i in others:
        assert s.result(i)["status"] == 0
    # the pair noise changes the trajectory: the same request without it differs
    s2 = Server()
    r2 = _pn_submit(s2, w, steps, 0.3, 0)
    s2.drain(120)
    assert rel_l2(s2.result(r2)["vel"], v) > 1e-2


def test_served_pair_noise_admission_counts_its_bytes():
    """Admission counts the pair-noise buffers exactly: a budget of the bytes
    a plain context holds after gld_set_pair_noise admits the request, one
    byte less refuses it (GLD_E_NOMEM); a pair kernel the Gershgorin bound
    refuses fails its request alone (GLD_E_NOT_PSD); a degree outside
    [0, 16] is refused at submission."""
    from paper_1808_00270_gb300 import GLDError, Server
    from paper_1808_00270_gb300.binding import E_INVAL, E_NOMEM, E_NOT_PSD
    w = _workload("pn_bytes", 1200, 0.1, 120, 61)
    held = _pn_plain(w, 0.3, 10).bytes()
    for budget, want in ((held, 0), (held - 1, E_NOMEM)):
        s = Server(hbm_budget=budget)
        i = _pn_submit(s, w, 70, 0.3, 10)
        s.drain(60)
        assert s.result(i)["status"] == want
        if want == 0:
            assert s.stats()["bytes_peak"] == held
    s = Server()
    bad = _pn_submit(s, w, 70, 1.0, 8)
    ok = _pn_submit(s, w, 70, 0.3, 8)
    s.drain(60)
    assert s.result(bad)["status"] == E_NOT_PSD and s.result(ok)["status"] == 0
    assert s.stats()["failed"] == 1 and s.stats()["bytes"] == 0
    for deg in (-1, 17):
        with pytest.raises(GLDError) as e:
            _pn_submit(s, w, 70, 0.3, deg)
        assert e.value.status == E_INVAL
