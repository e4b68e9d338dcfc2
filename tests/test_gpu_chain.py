"""The fused multi-layer chain kernel through the C ABI: against the single
step, against L separate single-step launches, and against the FP64 oracle's
chain on the 256-event workload (sampled; every track with KF_PARITY_FULL=1)."""
import ctypes
import os

import numpy as np
import pytest
import torch

import oracle
import parity_log
from oracle import compare
from paper_2401_14221_gb300 import build as kbuild
from paper_2401_14221_gb300 import kf
from paper_2401_14221_gb300 import workload as W

pytestmark = pytest.mark.gpu

VARIANT_FORM = {kf.KF_DF_UPDATE: oracle.FORM_STANDARD,
                kf.KF_FP32: oracle.FORM_STANDARD, kf.KF_FP64_UPDATE: oracle.FORM_STANDARD,
                kf.KF_JOSEPH: oracle.FORM_JOSEPH, kf.KF_FP64: oracle.FORM_STANDARD,
                kf.KF_ADAPTIVE: oracle.FORM_STANDARD}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    torch.cuda.set_device(0)
    yield torch.device("cuda:0")
    assert kf.kf_take_device_error() == 0


@pytest.fixture(scope="module")
def chain_full():
    return W.make_chain(events=256, seed=1)


def oracle_chain(cw, idx, form=oracle.FORM_STANDARD):
    hit = np.ascontiguousarray(cw.hit[:, :, idx].transpose(0, 2, 1), dtype=np.float64)
    hc = np.ascontiguousarray(cw.hitcov[:, :, idx].transpose(0, 2, 1), dtype=np.float64)
    return oracle.chain_batch(cw.kinds, cw.pos, cw.state.T[idx], cw.cov.T[idx], cw.charge[idx],
                              hit, hc, cw.bz, form, threads=8)


def ill_conditioned(cw, idx):
    """Tracks with a layer the FP32 step cannot resolve to the bounds, by the
    oracle's own arithmetic: a hit that shrinks a measured variance by more
    than 1e4, a cylinder crossed at |cos(incidence)| < 0.3, or an update that
    leaves 1/pT <= 0 (the criteria of KF_ADAPTIVE's marking pass)."""
    out = np.zeros(len(idx), dtype=bool)
    for k, i in enumerate(idx):
        p = cw.state[:, i].astype(np.float64)
        c21 = cw.cov[:, i].astype(np.float64)
        q = int(cw.charge[i])
        for l in range(cw.L):
            kind, pos = int(cw.kinds[l]), float(cw.pos[l])
            hit = cw.hit[l, :, i].astype(np.float64)
            hc = cw.hitcov[l, :, i].astype(np.float64)
            prop = oracle.propagate_to_z if kind == W.P2Z else oracle.propagate_to_r
            pp, J, st = prop(p, q, cw.bz, pos)
            if st:
                continue
            C = compare.unpack(c21[None])[0]
            Cp = J @ C @ J.T
            if kind == W.P2Z:
                s0, s1 = (Cp[0, 0] + hc[0]) / hc[0], (Cp[1, 1] + hc[2]) / hc[2]
                graz = False
            else:
                ph = np.arctan2(hit[1], hit[0])
                u = np.array([-np.sin(ph), np.cos(ph)])
                V = np.array([[hc[0], hc[1]], [hc[1], hc[2]]])
                v0 = u @ V @ u
                s0, s1 = (u @ Cp[:2, :2] @ u + v0) / v0, (Cp[2, 2] + hc[5]) / hc[5]
                graz = abs(pp[0] * np.cos(pp[4]) + pp[1] * np.sin(pp[4])) < 0.3 * pos
            if s0 > 1e4 or s1 > 1e4 or graz:
                out[k] = True
                break
            p, c21, _, _ = oracle.step(kind, p, c21, q, hit, hc, cw.bz, pos)
            if p[3] <= 0.0:
                out[k] = True
                break
    return out


def ends_on_cylinder(cw, o_st):
    """Tracks whose last reached layer is a cylinder (their covariance is
    compared in that surface's frame)."""
    r = np.hypot(o_st[:, 0], o_st[:, 1])
    on_plane = np.isin(o_st[:, 2], cw.pos[cw.kinds == W.P2Z].astype(np.float64))
    on_cyl = np.zeros(len(o_st), dtype=bool)
    for R in cw.pos[cw.kinds == W.P2R].astype(np.float64):
        on_cyl |= np.abs(r - R) <= 1e-5 * R
    return on_cyl & ~on_plane


@pytest.mark.parametrize("kind", [W.P2Z, W.P2R])
@pytest.mark.parametrize("layout", [(kf.KF_SOA, 0), (kf.KF_AOSOA, 32)])
@pytest.mark.parametrize("precision", [kf.KF_FP32, kf.KF_FP64, kf.KF_ADAPTIVE, kf.KF_DF_UPDATE])
def test_chain_of_one_layer_equals_single_step_bitwise(dev, kind, layout, precision):
    w = W.make_p2z(20011, seed=41) if kind == W.P2Z else W.make_p2r(1, 20011, seed=41)
    b = kf.upload(w, layout[0], layout[1], dev)
    b.run(precision)
    ref = b.download()
    cw = W.ChainWorkload(n=w.n, bz=w.bz, kinds=np.array([kind], dtype=np.int32),
                         pos=np.array([w.surf], dtype=np.float32), event_sizes=np.array([w.n]),
                         state=w.state, cov=w.cov, charge=w.charge, hit=w.hit[None],
                         hitcov=w.hitcov[None], truth_pool_layers=np.zeros((1, 6, 1)),
                         truth_index=np.zeros(w.n, dtype=np.int64))
    dc = kf.chain_upload(cw, layout[0], layout[1], dev)
    dc.run(precision)
    got = dc.download()
    for a, c in zip(ref, got):
        assert np.array_equal(a, c)


@pytest.mark.parametrize("precision", [kf.KF_FP32, kf.KF_JOSEPH, kf.KF_DF_UPDATE])
def test_chain_equals_per_layer_launches_bitwise(dev, precision):
    cw = W.make_chain(events=6, seed=42)
    dc = kf.chain_upload(cw, kf.KF_AOSOA, 32, dev)
    dc.run(precision)
    fused = dc.download()
    dc.reset()
    dc.run_plain(precision)
    plain = dc.download()
    assert np.array_equal(fused[0], plain[0]) and np.array_equal(fused[1], plain[1])


@pytest.mark.parametrize("precision", [kf.KF_FP32, kf.KF_ADAPTIVE])
def test_chain_on_page_locked_host_arrays(dev, precision):
    # the chain kernels reach page-locked host memory with plain loads and
    # stores (over the CPU-GPU link): same results as on device arrays
    cw = W.make_chain(events=4, seed=43)
    dc = kf.chain_upload(cw, kf.KF_AOSOA, 32, dev)
    dc.run(precision)
    ref = dc.download()
    pin = lambda t: t.cpu().pin_memory()
    st, cv, q = pin(dc.state0), pin(dc.cov0), pin(dc.charge)
    hits, hcs, status = pin(dc.hits), pin(dc.hit_covs), pin(torch.zeros_like(dc.status))
    rc = kf.load().kf_kalman_chain(
        ctypes.byref(kf.make_params(cw.bz, precision)), dc.layout, st.data_ptr(), cv.data_ptr(),
        q.data_ptr(), hits.data_ptr(), hcs.data_ptr(), dc.layers, cw.L, status.data_ptr(),
        torch.cuda.current_stream().cuda_stream)
    assert rc == kf.KF_OK, kf.kf_last_error_string()
    torch.cuda.synchronize()
    dc.state.copy_(st)
    dc.cov.copy_(cv)
    dc.status.copy_(status)
    got = dc.download()
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


@pytest.fixture(scope="module")
def chain_sample(chain_full):
    """Sampled tracks of the 256-event chain and which of them are
    ill-conditioned (by the oracle)."""
    n = chain_full.n
    idx = np.unique(np.concatenate([np.arange(200), np.linspace(0, n - 1, 3000).astype(np.int64),
                                    np.arange(n - 200, n)]))
    return idx, ill_conditioned(chain_full, idx)


@pytest.mark.parametrize("precision", [kf.KF_FP32, kf.KF_FP64_UPDATE, kf.KF_DF_UPDATE,
                                       kf.KF_JOSEPH, kf.KF_FP64,
                                       kf.KF_ADAPTIVE])
def test_chain_matches_oracle_on_256_events(dev, chain_full, chain_sample, precision):
    cw = chain_full
    dc = kf.chain_upload(cw, kf.KF_AOSOA, 32, dev)
    dc.run(precision)
    st, cv, stat = dc.download()
    float_state = precision in (kf.KF_FP32, kf.KF_FP64_UPDATE, kf.KF_DF_UPDATE, kf.KF_JOSEPH)
    if os.environ.get("KF_PARITY_FULL") == "1":
        # every track; for the float-state variants every track the adaptive
        # pass does not mark (those it marks are the ill-conditioned ones)
        idx = np.arange(cw.n)
        if float_state:
            dc.reset()
            dc.run(kf.KF_FP32)
            f32 = dc.download()
            dc.reset()
            dc.run(kf.KF_ADAPTIVE)
            ada = dc.download()
            marked = np.any(ada[0] != f32[0], axis=0) | np.any(ada[1] != f32[1], axis=0)
            assert 0 < marked.sum() < 0.01 * cw.n
            idx = idx[~marked]
    else:
        idx, ill = chain_sample
        if float_state:
            # float-state variants meet the bounds on well-conditioned tracks
            # only (about 0.6 % of this workload is ill-conditioned; KF_ADAPTIVE
            # and KF_FP64 are checked on every track)
            assert 0 < ill.sum() < 0.02 * len(idx)
            idx = idx[~ill]
    o_st, o_cv, o_stat = oracle_chain(cw, idx, VARIANT_FORM[precision])
    rep = compare.compare(st.T[idx], cv.T[idx], stat[idx], o_st, o_cv, o_stat,
                          on_cylinder=ends_on_cylinder(cw, o_st))
    parity_log.expect_ok("chain", rep)


def test_adaptive_chain_meets_the_bounds_on_every_track(dev, chain_full):
    # KF_ADAPTIVE is the variant that meets the bounds on every track: the
    # whole 256-event workload (about 1.96 M tracks, 15 layers, some crossing
    # the outer barrel layers at grazing incidence) against the oracle,
    # element by element, with no track left out.
    cw = chain_full
    dc = kf.chain_upload(cw, kf.KF_AOSOA, 32, dev)
    dc.run(kf.KF_ADAPTIVE)
    st, cv, stat = dc.download()
    idx = np.arange(cw.n)
    o_st, o_cv, o_stat = oracle_chain(cw, idx)
    rep = compare.compare(st.T, cv.T, stat, o_st, o_cv, o_stat,
                          on_cylinder=ends_on_cylinder(cw, o_st))
    assert rep["n"] == cw.n
    parity_log.expect_ok("chain", rep)


def test_adaptive_chain_in_a_cuda_graph(dev):
    # the adaptive chain captured into a CUDA graph (its second pass's list
    # becomes an allocation node of the graph) replays to the eager result,
    # bit for bit, twice
    cw = W.make_chain(events=16, seed=47)
    dc = kf.chain_upload(cw, kf.KF_AOSOA, 32, dev)
    dc.run(kf.KF_FP32)
    f32 = dc.download()
    dc.reset()
    dc.run(kf.KF_ADAPTIVE)
    ref = dc.download()
    assert np.any(ref[1] != f32[1])  # some tracks went through the second pass
    g = torch.cuda.CUDAGraph()
    dc.reset()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=torch.cuda.Stream()):
        dc.run(kf.KF_ADAPTIVE)
    for _ in range(2):
        dc.reset()
        g.replay()
        torch.cuda.synchronize()
        for x, y in zip(ref, dc.download()):
            assert np.array_equal(x, y)


def test_empty_chain_and_bad_layers(dev):
    cw = W.make_chain(events=1, seed=43, sizes=np.array([100]))
    dc = kf.chain_upload(cw, kf.KF_SOA, 0, dev)
    before = dc.state.clone()
    kf.kf_kalman_chain(kf.make_params(cw.bz), dc.layout, dc.state, dc.cov, dc.charge, dc.hits,
                       dc.hit_covs, kf.make_layers([], []))
    torch.cuda.synchronize()
    assert torch.equal(before, dc.state)
    bad = kf.make_layers([5], [30.0])
    with pytest.raises(kf.KfError) as e:
        kf.kf_kalman_chain(kf.make_params(cw.bz), dc.layout, dc.state, dc.cov, dc.charge,
                           dc.hits, dc.hit_covs, bad)
    assert e.value.code == kf.KF_ERR_ARG


def test_adaptive_chain_redo_pass(dev, chain_full):
    # KF_ADAPTIVE: the FP32 chain kernel gives up on a track at its first
    # ill-conditioned layer and leaves it (inputs untouched) to a second
    # kernel, which reruns the whole chain with the state in double.  Some
    # tracks of this workload barely reach the outer barrel layers and cross
    # them at grazing incidence (cos down to 0.004).
    cw = chain_full
    dc = kf.chain_upload(cw, kf.KF_AOSOA, 32, dev)
    dc.run(kf.KF_FP32)
    f32 = dc.download()
    dc.reset()
    dc.run(kf.KF_ADAPTIVE)
    ada = dc.download()
    assert not np.any(ada[2] & 0x80)
    redone = np.any(ada[1] != f32[1], axis=0)
    assert 0 < int(redone.sum()) < cw.n // 10
    # tracks no layer marked are bitwise the FP32 chain
    assert np.array_equal(ada[0][:, ~redone], f32[0][:, ~redone])
    # and the redone ones bitwise the all-FP64 chain (the second pass runs
    # the same double chain from the same inputs, in whatever order it
    # gathered them)
    dc.reset()
    dc.run(kf.KF_FP64)
    f64 = dc.download()
    for x, y in zip(ada, f64):
        assert np.array_equal(x[..., redone], y[..., redone])
    # the second pass per span instead of over one compacted list: the same
    kf.kf_set_chain_redo(kf.KF_CHAIN_REDO_SPAN)
    try:
        dc.reset()
        dc.run(kf.KF_ADAPTIVE)
        per_span = dc.download()
    finally:
        kf.kf_set_chain_redo(kf.KF_CHAIN_REDO_LIST)
    for x, y in zip(ada, per_span):
        assert np.array_equal(x, y)
    # the oracle on the redone tracks
    idx = np.flatnonzero(redone)
    o_st, o_cv, o_stat = oracle_chain(cw, idx, oracle.FORM_STANDARD)
    rep = compare.compare(ada[0].T[idx], ada[1].T[idx], ada[2][idx], o_st, o_cv, o_stat,
                          on_cylinder=ends_on_cylinder(cw, o_st))
    parity_log.expect_ok("chain", rep)
    # the status array is required
    with pytest.raises(kf.KfError) as e:
        kf.kf_kalman_chain(kf.make_params(cw.bz, kf.KF_ADAPTIVE), dc.layout, dc.state, dc.cov,
                           dc.charge, dc.hits, dc.hit_covs, dc.layers, None)
    assert e.value.code == kf.KF_ERR_ARG
