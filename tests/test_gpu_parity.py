"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Bounds (oracle/compare.py): relative error <= 1e-4 on track parameters
(floors for values near zero, phi as an angle) and <= 1e-3 on covariance
elements relative to sqrt(C_ii C_jj); per-track status bits must agree
exactly.  Full-size workloads run whole on the GPU and are checked on a
sample that always includes the first and last tracks (the ragged tail).
"""
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

LAYOUTS = [(kf.KF_SOA, 0), (kf.KF_AOSOA, 16), (kf.KF_AOSOA, 32), (kf.KF_AOSOA, 64),
           (kf.KF_AOSOA, 128)]
VARIANT_FORM = {kf.KF_FP32: oracle.FORM_STANDARD, kf.KF_FP64_UPDATE: oracle.FORM_STANDARD,
                kf.KF_JOSEPH: oracle.FORM_JOSEPH, kf.KF_FP64: oracle.FORM_STANDARD,
                kf.KF_ADAPTIVE: oracle.FORM_STANDARD, kf.KF_DF_UPDATE: oracle.FORM_STANDARD}
ALL_VARIANTS = [kf.KF_FP32, kf.KF_FP64_UPDATE, kf.KF_JOSEPH, kf.KF_FP64, kf.KF_ADAPTIVE,
                kf.KF_DF_UPDATE]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    torch.cuda.set_device(0)
    kf.kf_set_step_kernel(kf.KF_STEP_AUTO)
    yield torch.device("cuda:0")
    kf.kf_set_step_kernel(kf.KF_STEP_AUTO)
    # no bounded device wait gave up anywhere in this module
    assert kf.kf_take_device_error() == 0


@pytest.fixture(params=[kf.KF_STEP_DIRECT, kf.KF_STEP_STAGED], ids=["direct", "staged"])
def step_kernel(request, dev):
    kf.kf_set_step_kernel(request.param)
    yield request.param
    kf.kf_set_step_kernel(kf.KF_STEP_AUTO)


@pytest.fixture(params=[kf.KF_HOST_COPY, kf.KF_HOST_DIRECT], ids=["copy", "direct"])
def host_path(request, dev):
    """The host-array calls' data path: chunked copies through the workspace,
    or the kernel on the host arrays in place."""
    kf.kf_set_host_path(request.param)
    yield request.param
    kf.kf_set_host_path(kf.KF_HOST_AUTO)


def run_host_or_skip(hb, host_path, pinned, **kw):
    """hb.run(), skipping direct runs on pageable memory where the device
    cannot reach it (no host page-table access)."""
    try:
        hb.run(**kw)
    except kf.KfError as e:
        if host_path == kf.KF_HOST_DIRECT and not pinned and "not reachable" in str(e):
            pytest.skip("this device does not reach pageable host memory")
        raise


@pytest.fixture(scope="module")
def w_p2z():
    return W.single_step_p2z()


@pytest.fixture(scope="module")
def w_p2r():
    return W.single_step_p2r_paper_scale()


@pytest.fixture(scope="module")
def w_prec():
    return W.precision_p2z(), W.precision_p2r()


def sample_indices(n, k=20000):
    if n <= k:
        return np.arange(n)
    idx = np.concatenate([np.arange(256), np.linspace(0, n - 1, k).astype(np.int64),
                          np.arange(n - 256, n)])
    return np.unique(idx)


def oracle_on(w, idx, form=oracle.FORM_STANDARD, surf=None):
    if surf is None:
        surf = w.surf
    s = surf[idx] if np.ndim(surf) > 0 else surf
    return oracle.step_batch(w.kind, w.state.T[idx], w.cov.T[idx], w.charge[idx], w.hit.T[idx],
                             w.hitcov.T[idx], s, w.bz, form, threads=8)


def cylinder_frame(w, o_stat):
    """p2r: a track on the cylinder has no variance along the surface normal,
    so its covariance is compared in the surface frame (a Cartesian element
    such as C_xx = sin^2(a) C_tt is 1e-16 for a crossing near the x axis)."""
    return (np.asarray(o_stat) & oracle.NO_INTERSECT) == 0 if w.kind == W.P2R else None


def check(w, b, idx, form=oracle.FORM_STANDARD, surf=None, oracle_out=None):
    """Compare tracks idx of the batch's results with the oracle's (computed
    here, or given as oracle_out for exactly those tracks)."""
    st, cv, stat = b.download()
    # a bounded device wait that gave up leaves tiles unwritten: reported as
    # such, before any comparison
    parity_log.expect_no_device_error(n=w.n, layout=(b.layout.kind, b.layout.width))
    o_st, o_cv, o_stat, _ = oracle_out if oracle_out is not None else oracle_on(w, idx, form, surf)
    rep = compare.compare(st.T[idx], cv.T[idx], stat[idx], o_st, o_cv, o_stat,
                          on_cylinder=cylinder_frame(w, o_stat))
    # report track numbers in the batch, not in the sample
    for key in ("worst_param", "worst_cov"):
        if key in rep:
            rep[key]["batch_track"] = int(idx[rep[key]["track"]])
    return parity_log.expect_ok("step", rep, n=w.n, kind=w.kind,
                                layout=(b.layout.kind, b.layout.width), form=form)


def run(w, dev, layout=(kf.KF_SOA, 0), precision=kf.KF_FP32, surf=None):
    b = kf.upload(w, layout[0], layout[1], dev, surf)
    b.run(precision)
    torch.cuda.synchronize()
    return b


# ------------------------------------------------------------ workloads

@pytest.mark.parametrize("layout", LAYOUTS)
def test_p2z_single_step_8192(dev, w_p2z, layout, step_kernel):
    b = run(w_p2z, dev, layout)
    check(w_p2z, b, np.arange(w_p2z.n))


@pytest.fixture(scope="module")
def o_p2r_all(w_p2r):
    """The oracle on every track of the paper-scale p2r batch."""
    return oracle_on(w_p2r, np.arange(w_p2r.n))


@pytest.mark.parametrize("layout", LAYOUTS)
def test_p2r_paper_scale_960k(dev, w_p2r, o_p2r_all, layout, step_kernel):
    # the headline layout (AoSoA, W = 32): every one of the 960,000 tracks,
    # element by element, with both kernels; the other layouts on a sample
    # (test_staged_and_direct_kernels_agree_bitwise compares them in full)
    b = run(w_p2r, dev, layout)
    if layout == (kf.KF_AOSOA, 32):
        rep = check(w_p2r, b, np.arange(w_p2r.n), oracle_out=o_p2r_all)
        assert rep["n"] == w_p2r.n
    else:
        idx = sample_indices(w_p2r.n)
        rep = check(w_p2r, b, idx, oracle_out=tuple(x[idx] for x in o_p2r_all))
    assert rep["flagged"] == 0


@pytest.mark.parametrize("precision", ALL_VARIANTS)
def test_precision_study_pt_0p2_to_100(dev, w_prec, precision, step_kernel):
    # a sample of each million by default; every track with KF_PARITY_FULL=1
    full = os.environ.get("KF_PARITY_FULL") == "1"
    for w in w_prec:
        b = run(w, dev, (kf.KF_AOSOA, 32), precision)
        check(w, b, np.arange(w.n) if full else sample_indices(w.n), VARIANT_FORM[precision])


def test_adaptive_step_meets_the_bounds_on_every_track(dev, w_prec):
    # KF_ADAPTIVE on the whole precision study, 1,000,000 p2z and 1,000,000
    # p2r tracks with pT from 0.2 to 100 GeV, against the oracle on every
    # track (the other variants are compared on a sample above)
    for w in w_prec:
        b = run(w, dev, (kf.KF_AOSOA, 32), kf.KF_ADAPTIVE)
        rep = check(w, b, np.arange(w.n))
        assert rep["n"] == w.n


def test_double_float_update_carries_fp64_update_precision(dev, w_prec):
    # KF_DF_UPDATE and KF_FP64_UPDATE share the FP32 propagation and compute
    # S^-1, K and C'' far beyond FP32 (double-float about 48 bits, double 53)
    # before one rounding to FP32: their results must agree to a few FP32
    # ulps, much closer than the FP32 update comes to either.  A double-float
    # step that silently lost its low word would fail the first bound.
    for w in w_prec:
        outs = {p: run(w, dev, (kf.KF_AOSOA, 32), p).download()
                for p in (kf.KF_FP64_UPDATE, kf.KF_DF_UPDATE, kf.KF_FP32)}
        ref = outs[kf.KF_FP64_UPDATE]
        on_cyl = cylinder_frame(w, ref[2])

        def rep(o):
            return compare.compare(o[0].T, o[1].T, o[2], ref[0].T, ref[1].T, ref[2],
                                   on_cylinder=on_cyl)
        r_df, r_32 = rep(outs[kf.KF_DF_UPDATE]), rep(outs[kf.KF_FP32])
        assert r_df["status_equal"]
        assert r_df["param"]["max"] <= 5e-7 and r_df["cov"]["max"] <= 5e-7, r_df
        assert r_32["cov"]["max"] > 10 * r_df["cov"]["max"], (r_32["cov"], r_df["cov"])


@pytest.mark.parametrize("layout", LAYOUTS[1:])
@pytest.mark.parametrize("precision", ALL_VARIANTS)
def test_staged_and_direct_kernels_agree_bitwise(dev, w_p2r, layout, precision):
    # the kernels run the same per-track arithmetic; only the loads differ
    # (staged: 2 CTAs/SM x 3 stages and 3 CTAs/SM x 2 stages, the latter
    # compiled to 72 registers)
    outs = []
    for mode, ctas in ((kf.KF_STEP_DIRECT, 0), (kf.KF_STEP_STAGED, 2), (kf.KF_STEP_STAGED, 3)):
        kf.kf_set_step_kernel(mode)
        kf.kf_set_staged_ctas_per_sm(ctas)
        outs.append(run(w_p2r, dev, layout, precision).download())
    kf.kf_set_step_kernel(kf.KF_STEP_AUTO)
    kf.kf_set_staged_ctas_per_sm(0)
    for other in outs[1:]:
        for a, c in zip(outs[0], other):
            assert np.array_equal(a, c)


@pytest.mark.parametrize("ctas", [2, 3])
def test_staged_fp64_repeats_bitwise(dev, w_prec, ctas):
    # The staged kernel's all-FP64 variant on the precision study (the case
    # of the one parity failure never explained), launched again and again
    # on one stream into outputs poisoned with a NaN pattern before each
    # launch: every repeat gives the first one's bits, no output is left
    # unwritten, and the device error word stays clear.  A race between the
    # pipeline's copies and the warps that read them, or a wait that gave
    # up, would show as a difference between repeats.
    kf.kf_set_step_kernel(kf.KF_STEP_STAGED)
    kf.kf_set_staged_ctas_per_sm(ctas)
    try:
        for w in w_prec:
            b = kf.upload(w, kf.KF_AOSOA, 32, dev)
            runs = []
            for _ in range(6):
                b.state_out.fill_(float("nan"))
                b.cov_out.fill_(float("nan"))
                b.status.fill_(0xFF)
                b.run(kf.KF_FP64)
                torch.cuda.synchronize()
                parity_log.expect_no_device_error(case="staged FP64 repeat", ctas=ctas)
                st, cv, status = b.download()
                runs.append((np.ascontiguousarray(st, dtype=np.float32).view(np.uint32),
                             np.ascontiguousarray(cv, dtype=np.float32).view(np.uint32), status))
            assert not np.any(runs[0][2] == 0xFF)  # every status byte written
            for r in runs[1:]:
                for x, y in zip(runs[0], r):
                    assert np.array_equal(x, y)
    finally:
        kf.kf_set_step_kernel(kf.KF_STEP_AUTO)
        kf.kf_set_staged_ctas_per_sm(0)


# ----------------------------------------------------------- edge cases

@pytest.mark.parametrize("n", [1, 2, 4, 31, 33, 127, 129, 255, 257, 260, 1007, 4100, 77777])
@pytest.mark.parametrize("layout", [(kf.KF_SOA, 0), (kf.KF_AOSOA, 128), (kf.KF_AOSOA, 16)])
def test_ragged_sizes(dev, n, layout, step_kernel):
    for w in (W.make_p2z(n, seed=n), W.make_p2r(1, n, seed=n)):
        b = run(w, dev, layout)
        check(w, b, np.arange(n))


def test_empty_batch_launches_nothing(dev):
    w = W.make_p2z(16, seed=2)
    b = kf.upload(w, kf.KF_SOA, 0, dev)
    b.state_out.fill_(123.0)
    kf.kf_p2z_propagate_update(kf.make_params(w.bz), kf.make_layout(kf.KF_SOA, 0, 0), b.state_in,
                               b.cov_in, b.state_out, b.cov_out, b.charge, b.hit, b.hit_cov,
                               b.surf)
    torch.cuda.synchronize()
    assert torch.all(b.state_out == 123.0)


@pytest.mark.parametrize("kind", [W.P2Z, W.P2R])
def test_in_place_equals_out_of_place(dev, kind):
    w = W.make_p2z(5000, seed=5) if kind == W.P2Z else W.make_p2r(1, 5000, seed=5)
    b = run(w, dev, (kf.KF_AOSOA, 64))
    ref = b.download()
    b2 = kf.upload(w, kf.KF_AOSOA, 64, dev)
    b2.run(in_place=True)
    torch.cuda.synchronize()
    b2.state_out, b2.cov_out = b2.state_in, b2.cov_in
    got = b2.download()
    for a, c in zip(ref, got):
        assert np.array_equal(a, c)


@pytest.mark.parametrize("precision", [kf.KF_ADAPTIVE, kf.KF_FP64])
def test_per_track_surfaces(dev, step_kernel, precision):
    # every track has its own plane / cylinder and its hit lies on it
    rng = np.random.default_rng(8)
    zs = rng.uniform(20.0, 120.0, 3001)
    w = W.make_p2z(3001, seed=8, zt=zs)
    b = run(w, dev, (kf.KF_SOA, 0), precision)
    check(w, b, np.arange(w.n))
    # Cylinders out to 150 cm: low-pT tracks reach them after long paths,
    # some at grazing incidence, where the hit shrinks the propagated
    # variance by up to ~1e6.  There the FP32 covariance update loses more
    # digits than FP32 holds; KF_ADAPTIVE redoes those tracks in FP64.
    # Covariances of tracks on the cylinder are compared in its surface frame.
    # 2 rho = 88..175 cm for pT 0.5..1 GeV: some never get there
    w = grazing_p2r()
    b = run(w, dev, (kf.KF_AOSOA, 32), precision)
    st, cv, stat = b.download()
    o_st, o_cv, o_stat, _ = oracle_on(w, np.arange(w.n))
    on_cyl = (o_stat & oracle.NO_INTERSECT) == 0
    rep = compare.compare(st.T, cv.T, stat, o_st, o_cv, o_stat, on_cylinder=on_cyl)
    parity_log.expect_ok("step", rep)
    assert rep["flagged"] > 0 and rep["flagged"] == int(np.sum(~w.reached))


def grazing_p2r(seed=9, n=3001):
    # cylinders out to 150 cm: low-pT tracks cross some at grazing incidence
    rs = np.random.default_rng(seed).uniform(5.0, 150.0, n)
    return W.make_p2r(1, n, seed=seed, R=rs)


@pytest.mark.parametrize("layout", [(kf.KF_SOA, 0), (kf.KF_AOSOA, 16)])
def test_adaptive_redo_pass_in_place(dev, step_kernel, layout):
    # KF_ADAPTIVE marks ill-conditioned tracks in the FP32 kernel and redoes
    # them in a second kernel from the untouched inputs; in place the FP32
    # kernel must therefore leave those tracks' inputs alone.
    w = grazing_p2r()
    ref = run(w, dev, layout, kf.KF_ADAPTIVE).download()
    fp32 = run(w, dev, layout, kf.KF_FP32).download()
    b = kf.upload(w, layout[0], layout[1], dev)
    b.run(kf.KF_ADAPTIVE, in_place=True)
    torch.cuda.synchronize()
    b.state_out, b.cov_out = b.state_in, b.cov_in
    got = b.download()
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)
    # the redo pass ran: some tracks differ from FP32, and no mark is left
    redone = np.any(ref[1] != fp32[1], axis=0) & ((ref[2] & kf.NO_INTERSECT) == 0)
    assert 0 < int(redone.sum()) < w.n // 2
    assert not np.any(ref[2] & 0x80)


def test_adaptive_with_unaligned_status(dev):
    # the redo pass reads status 16 bytes at a time where it can, byte by
    # byte where the array is not 16-byte aligned or at its ragged end
    w = grazing_p2r()
    b = run(w, dev, (kf.KF_SOA, 0), kf.KF_ADAPTIVE)
    ref = b.download()
    big = torch.zeros(w.n + 16, dtype=torch.uint8, device=dev)
    status = big[3:3 + w.n]
    so, co = torch.empty_like(b.state_out), torch.empty_like(b.cov_out)
    kf.kf_p2r_propagate_update(kf.make_params(w.bz, kf.KF_ADAPTIVE), b.layout, b.state_in,
                               b.cov_in, so, co, b.charge, b.hit, b.hit_cov, b.surf, 1, status)
    torch.cuda.synchronize()
    assert torch.equal(so, b.state_out) and torch.equal(co, b.cov_out)
    assert np.array_equal(status.cpu().numpy(), ref[2])


def test_adaptive_needs_a_status_array(dev):
    w = W.make_p2r(1, 256, seed=5)
    b = kf.upload(w, kf.KF_AOSOA, 32, dev)
    b.state_out.fill_(7.0)
    with pytest.raises(kf.KfError) as e:
        kf.kf_p2r_propagate_update(kf.make_params(w.bz, kf.KF_ADAPTIVE), b.layout, b.state_in,
                                   b.cov_in, b.state_out, b.cov_out, b.charge, b.hit, b.hit_cov,
                                   b.surf, 0, None, None)
    assert e.value.code == kf.KF_ERR_ARG
    torch.cuda.synchronize()
    assert torch.all(b.state_out == 7.0)


def test_degenerate_tracks(dev, step_kernel):
    # unreachable cylinder, start outside, parallel to the plane, k = 0,
    # a non-positive-definite hit covariance
    w = W.make_p2r(1, 64, seed=10)
    w.state[3, 0:8] = 1.0 / 0.2          # pT 0.2 GeV: rho 17.5 cm, just reaches r = 30
    w.state[3, 8:16] = 1.0 / 0.1         # rho 8.8 cm: never reaches r = 30
    w.state[0, 16:24] = 35.0             # starts outside
    w.state[3, 24:32] = 0.0              # infinite momentum: straight line
    w.hitcov[5, 32:40] = -1.0            # S not positive definite
    b = run(w, dev)
    rep = check(w, b, np.arange(w.n))
    st = b.download()[2]
    assert np.all(st[8:24] & kf.NO_INTERSECT) and np.all(st[32:40] & kf.S_NOT_PD)
    assert rep["flagged"] >= 24
    w = W.make_p2z(64, seed=11)
    w.state[5, 0:8] = np.float32(np.pi / 2)  # parallel to the plane
    w.state[3, 8:16] = 0.0
    w.hitcov[0, 16:24] = -1.0
    b = run(w, dev)
    check(w, b, np.arange(w.n))
    st = b.download()[2]
    assert np.all(st[0:8] == kf.NO_INTERSECT) and np.all(st[16:24] & kf.S_NOT_PD)


def test_offsets_beyond_2_to_31_elements(dev):
    # 105M tracks: the covariance array holds > 2^31 floats, so element
    # offsets need 64-bit arithmetic.  The batch repeats a 1M-track workload.
    base = W.make_p2r(100, 10000, seed=12)
    reps = 105
    n = base.n * reps
    lay = kf.make_layout(kf.KF_SOA, 0, n)

    def rep_dev(a, dtype=torch.float32):
        t = torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        return t.repeat(1, reps).reshape(-1).contiguous() if t.dim() == 2 else t.repeat(reps)

    st_in, cv_in = rep_dev(base.state), rep_dev(base.cov)
    st_out, cv_out = torch.empty_like(st_in), torch.empty_like(cv_in)
    status = torch.zeros(n, dtype=torch.uint8, device=dev)
    kf.kf_p2r_propagate_update(kf.make_params(base.bz), lay, st_in, cv_in, st_out, cv_out,
                               rep_dev(base.charge), rep_dev(base.hit), rep_dev(base.hitcov),
                               torch.tensor([base.surf], device=dev), 0, status)
    torch.cuda.synchronize()
    idx = np.concatenate([np.arange(n - 3000, n), np.arange(0, n, n // 3000)])
    gi = torch.from_numpy(idx).to(dev)
    g_st = st_out.view(6, n)[:, gi].cpu().numpy().T
    g_cv = cv_out.view(21, n)[:, gi].cpu().numpy().T
    g_stat = status[gi].cpu().numpy()
    bi = idx % base.n
    o_st, o_cv, o_stat, _ = oracle_on(base, bi)
    rep = compare.compare(g_st, g_cv, g_stat, o_st, o_cv, o_stat,
                          on_cylinder=cylinder_frame(base, o_stat))
    parity_log.expect_ok("step", rep)
    del st_in, cv_in, st_out, cv_out
    torch.cuda.empty_cache()


# --------------------------------------------------- argument refusal

def test_bad_pointers_are_refused_not_launched(dev):
    w = W.make_p2z(1000, seed=13)
    b = kf.upload(w, kf.KF_SOA, 0, dev)
    p = kf.make_params(w.bz)
    lay = kf.make_layout(kf.KF_SOA, 0, w.n)
    args = [b.state_in, b.cov_in, b.state_out, b.cov_out, b.charge, b.hit, b.hit_cov, b.surf]

    def call(**over):
        a = list(args)
        for k, v in over.items():
            a[int(k[1:])] = v
        return kf.load().kf_p2z_propagate_update(
            ctypes.byref(p), lay, *[t if isinstance(t, int) else t.data_ptr() for t in a], 0, None,
            torch.cuda.current_stream().cuda_stream)

    host = np.zeros(21 * w.n, dtype=np.float32)
    assert call(a1=host.ctypes.data) == kf.KF_ERR_ARG          # pageable host memory
    assert call(a2=b.state_out.data_ptr() + 4) == kf.KF_ERR_ARG  # misaligned
    assert call(a2=b.state_in.data_ptr() + 16) == kf.KF_ERR_ARG  # partial overlap with state_in
    torch.cuda.synchronize()
    assert kf.kf_last_error_string() != ""


def test_short_buffer_is_refused(dev):
    # A buffer from its own cudaMalloc, smaller than the layout needs.
    w = W.make_p2z(4096, seed=14)
    b = kf.upload(w, kf.KF_SOA, 0, dev)
    n_big = 1 << 22  # 4M tracks need 100 MB of covariance: more than any segment holds here
    p = kf.make_params(w.bz)
    rc = kf.load().kf_p2z_propagate_update(
        ctypes.byref(p), kf.make_layout(kf.KF_SOA, 0, n_big), b.state_in.data_ptr(),
        b.cov_in.data_ptr(), b.state_out.data_ptr(), b.cov_out.data_ptr(), b.charge.data_ptr(),
        b.hit.data_ptr(), b.hit_cov.data_ptr(), b.surf.data_ptr(), 0, None,
        torch.cuda.current_stream().cuda_stream)
    assert rc == kf.KF_ERR_ARG
    assert "allocation" in kf.kf_last_error_string()


# ------------------------------------------------ host-array entry point

@pytest.mark.parametrize("layout", [(kf.KF_SOA, 0), (kf.KF_AOSOA, 64)])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_array_entry_matches_device_entry(dev, layout, pinned, host_path):
    # Copy path: 99,999 tracks in chunks of 16,384, seven chunks over both
    # pipeline slots, the last one ragged.  Direct path: the kernel reads and
    # writes the host arrays in place (page-locked, or pageable through the
    # host page tables).  The arithmetic is the same, so results are bitwise
    # equal to the device entry's.
    for w in (W.make_p2r(3, 33333, seed=15), W.make_p2z(99999, seed=16)):
        hb = kf.host_upload(w, layout[0], layout[1], dev, chunk_tracks=16384, pinned=pinned)
        run_host_or_skip(hb, host_path, pinned)
        torch.cuda.synchronize()
        got = hb.download()
        ref = run(w, dev, layout).download()
        for a, c in zip(ref, got):
            assert np.array_equal(a, c)
        idx = sample_indices(w.n, 4000)
        o_st, o_cv, o_stat, _ = oracle_on(w, idx)
        rep = compare.compare(got[0].T[idx], got[1].T[idx], got[2][idx], o_st, o_cv, o_stat,
                              on_cylinder=cylinder_frame(w, o_stat))
        parity_log.expect_ok("step", rep)


@pytest.mark.parametrize("n", [1, 33, 4097, 300001])
@pytest.mark.parametrize("layout", [(kf.KF_SOA, 0), (kf.KF_AOSOA, 128)])
def test_host_entry_default_chunk(dev, n, layout, host_path):
    # the default chunk (262,144 tracks): one chunk, or two with the last
    # one ragged; and the same sizes in place
    w = W.make_p2r(1, n, seed=18)
    hb = kf.host_upload(w, layout[0], layout[1], dev, pinned=True)
    hb.run()
    torch.cuda.synchronize()
    got = hb.download()
    ref = run(w, dev, layout).download()
    for a, c in zip(ref, got):
        assert np.array_equal(a, c)


@pytest.mark.parametrize("entry", ["workspace", "noalloc"])
def test_host_entries_run_adaptive_without_a_status_array(dev, entry, host_path):
    # KF_ADAPTIVE needs a status array on the device for its redo pass; the
    # host-array entry points use their own staging for it (on the direct
    # path: the workspace, or the no-allocation call's staging buffer), so
    # the caller may pass none.  Results equal the device entry's bit for bit.
    w = grazing_p2r()
    lay = (kf.KF_AOSOA, 32)
    ref = run(w, dev, lay, kf.KF_ADAPTIVE).download()
    hb = kf.host_upload(w, lay[0], lay[1], dev, chunk_tracks=1024, pinned=True)
    hb.state_out.fill_(np.nan)
    params = kf.make_params(w.bz, kf.KF_ADAPTIVE)
    if entry == "workspace":
        kf.kf_p2r_propagate_update_host(params, hb.layout, hb.state_in, hb.cov_in, hb.state_out,
                                        hb.cov_out, hb.charge, hb.hit, hb.hit_cov, hb.surf, 1,
                                        None, hb.workspace, 1024)
    else:
        kf.kf_propagate_update_host_noalloc(kf.KF_P2R, params, hb.layout, hb.state_in,
                                            hb.cov_in, hb.state_out, hb.cov_out, hb.charge,
                                            hb.hit, hb.hit_cov, hb.surf, 1, None, 1024)
    torch.cuda.synchronize()
    got = hb.download()
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_host_entry_rejects_small_workspace(dev):
    w = W.make_p2z(5000, seed=17)
    hb = kf.host_upload(w, kf.KF_SOA, 0, dev, chunk_tracks=1024)
    hb.workspace = hb.workspace[: hb.workspace.numel() // 2]
    kf.kf_set_host_path(kf.KF_HOST_COPY)
    try:
        with pytest.raises(kf.KfError) as e:
            hb.run()
        assert e.value.code == kf.KF_ERR_ARG
    finally:
        kf.kf_set_host_path(kf.KF_HOST_AUTO)


@pytest.mark.parametrize("precision", [kf.KF_FP32, kf.KF_JOSEPH, kf.KF_FP64, kf.KF_ADAPTIVE])
def test_host_direct_path_needs_no_workspace(dev, precision):
    # In place on page-locked memory the call needs no device memory at all
    # (KF_ADAPTIVE with its status array given).  Results equal the device
    # entry's bit for bit, for every precision variant.
    w = grazing_p2r() if precision == kf.KF_ADAPTIVE else W.make_p2r(2, 5001, seed=31)
    lay = (kf.KF_AOSOA, 32)
    ref = run(w, dev, lay, precision).download()
    hb = kf.host_upload(w, lay[0], lay[1], dev, pinned=True)
    hb.workspace = None
    kf.kf_set_host_path(kf.KF_HOST_DIRECT)
    try:
        hb.run(precision)
        torch.cuda.synchronize()
    finally:
        kf.kf_set_host_path(kf.KF_HOST_AUTO)
    got = hb.download()
    for a, c in zip(ref, got):
        assert np.array_equal(a, c)


def test_host_direct_path_refusals(dev):
    w = W.make_p2r(1, 4096, seed=32)
    lay = (kf.KF_SOA, 0)
    hb = kf.host_upload(w, lay[0], lay[1], dev, pinned=True)
    params = kf.make_params(w.bz, kf.KF_ADAPTIVE)
    kf.kf_set_host_path(kf.KF_HOST_DIRECT)
    try:
        # KF_ADAPTIVE without a status array and without a workspace: no
        # device memory for the redo marks
        with pytest.raises(kf.KfError) as e:
            kf.kf_p2r_propagate_update_host(params, hb.layout, hb.state_in, hb.cov_in,
                                            hb.state_out, hb.cov_out, hb.charge, hb.hit,
                                            hb.hit_cov, hb.surf, 1, None, None, 0)
        assert e.value.code == kf.KF_ERR_ARG
        # a page-locked array shorter than the layout needs (registered with
        # its exact extent: 1,024 floats where 21 x 4,096 are needed)
        short = np.zeros(1024, dtype=np.float32)
        cudart = torch.cuda.cudart()
        assert cudart.cudaHostRegister(short.ctypes.data, short.nbytes, 0) == \
            cudart.cudaError.success
        try:
            with pytest.raises(kf.KfError) as e:
                kf.kf_p2r_propagate_update_host(
                    kf.make_params(w.bz), hb.layout, hb.state_in, short.ctypes.data,
                    hb.state_out, hb.cov_out, hb.charge, hb.hit, hb.hit_cov, hb.surf, 1,
                    hb.status, None, 0)
            assert e.value.code == kf.KF_ERR_ARG
            assert "allocation" in kf.kf_last_error_string()
        finally:
            cudart.cudaHostUnregister(short.ctypes.data)
        # a misaligned float array cannot be read in place
        with pytest.raises(kf.KfError) as e:
            kf.kf_p2r_propagate_update_host(
                kf.make_params(w.bz), hb.layout, hb.state_in.data_ptr() + 2, hb.cov_in,
                hb.state_out, hb.cov_out, hb.charge, hb.hit, hb.hit_cov, hb.surf, 1, hb.status,
                None, 0)
        assert e.value.code == kf.KF_ERR_ARG
    finally:
        kf.kf_set_host_path(kf.KF_HOST_AUTO)
    torch.cuda.synchronize()


def test_device_entry_on_page_locked_arrays(dev):
    # Page-locked host arrays given to the device-array entry run the
    # one-thread-per-track kernel (plain loads), whatever kernel mode is set;
    # results equal those on device arrays bit for bit.
    w = W.make_p2r(2, 4100, seed=33)
    lay = (kf.KF_AOSOA, 32)
    ref = run(w, dev, lay).download()
    hb = kf.host_upload(w, lay[0], lay[1], dev, pinned=True)
    p = kf.make_params(w.bz)
    kf.kf_set_step_kernel(kf.KF_STEP_STAGED)
    try:
        rc = kf.load().kf_p2r_propagate_update(
            ctypes.byref(p), hb.layout, *[t.data_ptr() for t in (
                hb.state_in, hb.cov_in, hb.state_out, hb.cov_out, hb.charge, hb.hit, hb.hit_cov,
                hb.surf)], int(hb.surf.numel() > 1), hb.status.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
        assert rc == kf.KF_OK, kf.kf_last_error_string()
        torch.cuda.synchronize()
    finally:
        kf.kf_set_step_kernel(kf.KF_STEP_AUTO)
    got = hb.download()
    for a, c in zip(ref, got):
        assert np.array_equal(a, c)


# -------------------------------------------- compressed covariance store

@pytest.mark.parametrize("layout", [(kf.KF_SOA, 0), (kf.KF_AOSOA, 32)])
def test_compressed_covariance_step(dev, w_prec, layout):
    # FP32 sigmas + FP16 correlations in and out.  Against the oracle run on
    # the decoded input, the result is within the parity bounds; the FP16
    # encoding of the output adds at most 2^-12 of the correlation scale.
    for w in w_prec:
        lay = kf.make_layout(layout[0], layout[1], w.n)
        sig, rho = W.compress_cov(w.cov)
        st_in = kf.to_device(w.state, lay, dev)
        sg_in = kf.to_device(sig, lay, dev)
        rh_in = kf.to_device_rho(rho, lay, dev)
        st_out, sg_out, rh_out = torch.empty_like(st_in), torch.empty_like(sg_in), torch.empty_like(rh_in)
        status = torch.zeros(w.n, dtype=torch.uint8, device=dev)
        kind = kf.KF_P2Z if w.kind == W.P2Z else kf.KF_P2R
        kf.kf_propagate_update_compressed(
            kind, kf.make_params(w.bz), lay, st_in, sg_in, rh_in, st_out, sg_out, rh_out,
            torch.from_numpy(w.charge).to(dev), kf.to_device(w.hit, lay, dev),
            kf.to_device(w.hitcov, lay, dev), torch.tensor([w.surf], device=dev), 0, status)
        torch.cuda.synchronize()
        g_st = kf.from_device(st_out, 6, w.n, lay)
        g_sig = kf.from_device(sg_out, 6, w.n, lay)
        rh = kf.from_device_rho(rh_out, w.n, lay)
        g_cov = W.decompress_cov(g_sig, rh)
        # a sample by default; every track with KF_PARITY_FULL=1
        idx = np.arange(w.n) if os.environ.get("KF_PARITY_FULL") == "1" else sample_indices(w.n)
        c_in = W.decompress_cov(sig, rho)
        o_st, o_cv, o_stat, _ = oracle.step_batch(w.kind, w.state.T[idx], c_in.T[idx],
                                                  w.charge[idx], w.hit.T[idx], w.hitcov.T[idx],
                                                  w.surf, w.bz, threads=8)
        rep = compare.compare(g_st.T[idx], g_cov.T[idx], status.cpu().numpy()[idx], o_st, o_cv,
                              o_stat, on_cylinder=cylinder_frame(w, o_stat))
        parity_log.expect_ok("step", rep)


def run_compressed(w, dev, layout, precision, in_place=False):
    lay = kf.make_layout(layout[0], layout[1], w.n)
    sig, rho = W.compress_cov(w.cov)
    st_in = kf.to_device(w.state, lay, dev)
    sg_in = kf.to_device(sig, lay, dev)
    rh_in = kf.to_device_rho(rho, lay, dev)
    if in_place:
        st_out, sg_out, rh_out = st_in, sg_in, rh_in
    else:
        st_out, sg_out, rh_out = (torch.empty_like(st_in), torch.empty_like(sg_in),
                                  torch.empty_like(rh_in))
    status = torch.zeros(w.n, dtype=torch.uint8, device=dev)
    kind = kf.KF_P2Z if w.kind == W.P2Z else kf.KF_P2R
    per_track = np.ndim(w.surf) > 0
    surf = torch.from_numpy(np.atleast_1d(np.asarray(w.surf, dtype=np.float32))).to(dev)
    kf.kf_propagate_update_compressed(
        kind, kf.make_params(w.bz, precision), lay, st_in, sg_in, rh_in, st_out, sg_out, rh_out,
        torch.from_numpy(w.charge).to(dev), kf.to_device(w.hit, lay, dev),
        kf.to_device(w.hitcov, lay, dev), surf, int(per_track), status)
    torch.cuda.synchronize()
    g_st = kf.from_device(st_out, 6, w.n, lay)
    g_sig = kf.from_device(sg_out, 6, w.n, lay)
    rh = kf.from_device_rho(rh_out, w.n, lay)
    return g_st, W.decompress_cov(g_sig, rh), status.cpu().numpy()


def test_compressed_adaptive_redo_pass(dev):
    # the compressed store with KF_ADAPTIVE on grazing crossings: marked
    # tracks are decoded again from their untouched inputs and redone in
    # FP64, in place as out of place; the result is within the bounds
    w = grazing_p2r()
    lay = (kf.KF_AOSOA, 32)
    g = run_compressed(w, dev, lay, kf.KF_ADAPTIVE)
    g2 = run_compressed(w, dev, lay, kf.KF_ADAPTIVE, in_place=True)
    f32 = run_compressed(w, dev, lay, kf.KF_FP32)
    for x, y in zip(g, g2):
        assert np.array_equal(x, y)
    assert np.any(g[1] != f32[1]) and not np.any(g[2] & 0x80)
    sig, rho = W.compress_cov(w.cov)
    c_in = W.decompress_cov(sig, rho)
    o_st, o_cv, o_stat, _ = oracle.step_batch(w.kind, w.state.T, c_in.T, w.charge, w.hit.T,
                                              w.hitcov.T, w.surf, w.bz, threads=8)
    on_cyl = (o_stat & oracle.NO_INTERSECT) == 0
    rep = compare.compare(g[0].T, g[1].T, g[2], o_st, o_cv, o_stat, on_cylinder=on_cyl)
    parity_log.expect_ok("step", rep)


@pytest.mark.parametrize("precision", [kf.KF_FP32, kf.KF_JOSEPH, kf.KF_ADAPTIVE])
@pytest.mark.parametrize("kind", [W.P2Z, W.P2R])
def test_compressed_staged_equals_direct_bitwise(dev, kind, precision):
    # AoSoA: the staged compressed kernel; KF_STEP_DIRECT forces the one-
    # thread-per-track one.  Same arithmetic, same bits (ragged n).
    w = W.make_p2z(30011, seed=71) if kind == W.P2Z else grazing_p2r(seed=72, n=30011)
    lay = (kf.KF_AOSOA, 64)
    kf.kf_set_step_kernel(kf.KF_STEP_AUTO)
    staged = run_compressed(w, dev, lay, precision)
    kf.kf_set_step_kernel(kf.KF_STEP_DIRECT)
    try:
        direct = run_compressed(w, dev, lay, precision)
    finally:
        kf.kf_set_step_kernel(kf.KF_STEP_AUTO)
    for x, y in zip(staged, direct):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("width", [16, 32, 128])
def test_compressed_staged_equals_direct_bitwise_every_width(dev, width):
    # the staged kernel addresses a tile's correlation pairs from the tile's
    # first block, the one-thread-per-track kernel from the track index:
    # the same bits at every AoSoA width (ragged n)
    w = grazing_p2r(seed=73, n=20011)
    lay = (kf.KF_AOSOA, width)
    kf.kf_set_step_kernel(kf.KF_STEP_AUTO)
    staged = run_compressed(w, dev, lay, kf.KF_FP32)
    kf.kf_set_step_kernel(kf.KF_STEP_DIRECT)
    try:
        direct = run_compressed(w, dev, lay, kf.KF_FP32)
    finally:
        kf.kf_set_step_kernel(kf.KF_STEP_AUTO)
    for x, y in zip(staged, direct):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("n", [1, 129, 4099])
@pytest.mark.parametrize("layout", [(kf.KF_SOA, 0), (kf.KF_AOSOA, 16), (kf.KF_AOSOA, 128)])
def test_compressed_ragged_against_the_oracle(dev, layout, n):
    # odd track counts: SoA pair rows of odd length, a last AoSoA block
    # mostly padding, a single track; every track against the oracle on the
    # decoded input
    w = W.make_p2r(1, n, seed=74, pt_range=(0.2, 100.0))
    g = run_compressed(w, dev, layout, kf.KF_FP32)
    sig, rho = W.compress_cov(w.cov)
    c_in = W.decompress_cov(sig, rho)
    o_st, o_cv, o_stat, _ = oracle.step_batch(w.kind, w.state.T, c_in.T, w.charge, w.hit.T,
                                              w.hitcov.T, w.surf, w.bz, threads=8)
    rep = compare.compare(g[0].T, g[1].T, g[2], o_st, o_cv, o_stat,
                          on_cylinder=cylinder_frame(w, o_stat))
    parity_log.expect_ok("step", rep)


def test_compressed_bad_arguments_are_refused(dev):
    # a correlation array 4 bytes off the 16-byte rule, and an output that
    # partially overlaps its input, are refused on the host before a launch
    w = W.make_p2r(1, 1000, seed=15)
    lay = kf.make_layout(kf.KF_AOSOA, 32, w.n)
    sig, rho = W.compress_cov(w.cov)
    rh = kf.to_device_rho(rho, lay, dev)
    big = torch.zeros(2 * rh.numel(), dtype=torch.float16, device=dev)
    big[:rh.numel()] = rh
    st_in, sg_in = kf.to_device(w.state, lay, dev), kf.to_device(sig, lay, dev)
    st_out, sg_out = torch.empty_like(st_in), torch.empty_like(sg_in)
    rest = [torch.from_numpy(w.charge).to(dev), kf.to_device(w.hit, lay, dev),
            kf.to_device(w.hitcov, lay, dev), torch.tensor([w.surf], device=dev)]
    p = kf.make_params(w.bz)

    def call(rho_in, rho_out):
        ptrs = [st_in, sg_in, rho_in, st_out, sg_out, rho_out, *rest]
        return kf.load().kf_propagate_update_compressed(
            kf.KF_P2R, ctypes.byref(p), lay, *[t.data_ptr() for t in ptrs], 0, None,
            torch.cuda.current_stream().cuda_stream)

    n = rh.numel()
    assert call(big[2:2 + n], big[n:]) == kf.KF_ERR_ARG   # 4 bytes off alignment
    assert "aligned" in kf.kf_last_error_string()
    assert call(big[:n], big[8:8 + n]) == kf.KF_ERR_ARG   # 16 bytes into the input
    assert "overlap" in kf.kf_last_error_string()
    assert call(big[:n], big[n:]) == kf.KF_OK
    torch.cuda.synchronize()
    assert kf.kf_take_device_error() == 0


def test_prepared_step_equals_the_plain_call(dev):
    # the binding's prepared call marshals the arguments once; the launches
    # are the same calls, so the results are the same bits, on the current
    # stream and on another one
    w = W.make_p2z(8192, seed=1)
    b = kf.upload(w, kf.KF_AOSOA, 32, dev)
    b.run()
    torch.cuda.synchronize()
    ref = b.download()
    b.state_out.fill_(float("nan"))
    b.cov_out.fill_(float("nan"))
    step = b.prepare()
    step()
    torch.cuda.synchronize()
    for x, y in zip(ref, b.download()):
        assert np.array_equal(x, y)
    b.state_out.fill_(float("nan"))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        step(stream=s)
    s.synchronize()
    for x, y in zip(ref, b.download()):
        assert np.array_equal(x, y)
