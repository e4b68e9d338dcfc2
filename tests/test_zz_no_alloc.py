"""kf_propagate_update_host_noalloc against the workspace host-array entry point.

The no-allocation entry point is for callers that may not call cudaMalloc (a
plugin whose host process owns the device allocator, or a latency-critical
loop where an allocation would synchronise the device): it stages host
arrays through a fixed device buffer held by the library instead of a
caller-provided workspace.  Both entry points run the same kernel
arithmetic, so its results must equal kf_p2r/p2z_propagate_update_host's
bit for bit (state, covariance and status), call after call, while every
call reuses the same staging buffer; and a run of calls must leave the
device's free memory unchanged.  This file is collected last so that a run
stopping at the first failure has run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2401_14221_gb300 import build as kbuild
from paper_2401_14221_gb300 import kf
from paper_2401_14221_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kbuild.build()
    torch.cuda.set_device(0)
    return torch.device("cuda:0")


@pytest.fixture(params=[kf.KF_HOST_COPY, kf.KF_HOST_DIRECT], ids=["copy", "direct"])
def host_path(request, dev):
    """Staged through the library's buffer, or the kernel on the host arrays
    in place (the buffer unused)."""
    kf.kf_set_host_path(request.param)
    yield request.param
    kf.kf_set_host_path(kf.KF_HOST_AUTO)


def _noalloc(hb, fill, precision=kf.KF_FP32):
    """Run the no-allocation call on the host arrays of `hb`, writing into
    fresh host outputs pre-filled with `fill` (status with 255); returns SoA
    results."""
    st_out = torch.full_like(hb.state_out, fill)
    cv_out = torch.full_like(hb.cov_out, fill)
    status = torch.full_like(hb.status, 255)
    kind = kf.KF_P2Z if hb.kind == W.P2Z else kf.KF_P2R
    kf.kf_propagate_update_host_noalloc(
        kind, kf.make_params(hb.bz, precision), hb.layout, hb.state_in, hb.cov_in, st_out,
        cv_out, hb.charge, hb.hit, hb.hit_cov, hb.surf, int(hb.surf.numel() > 1), status)
    torch.cuda.synchronize()
    saved = hb.state_out, hb.cov_out, hb.status
    hb.state_out, hb.cov_out, hb.status = st_out, cv_out, status
    out = hb.download()
    hb.state_out, hb.cov_out, hb.status = saved
    return out


def _assert_equal(got, ref):
    # the same kernel arithmetic on the same inputs: bit for bit
    for name, g, r in zip(("state", "cov", "status"), got, ref):
        assert np.array_equal(g, r), f"{name} differs from the workspace entry point"


def _grazing_p2r(n=40001, seed=25):
    # cylinders out to 150 cm: some low-pT tracks cross them at grazing
    # incidence, so KF_ADAPTIVE redoes them in FP64 (through the status array)
    rs = np.random.default_rng(seed).uniform(5.0, 150.0, n)
    return W.make_p2r(1, n, seed=seed, R=rs)


@pytest.mark.parametrize("layout", [(kf.KF_SOA, 0), (kf.KF_AOSOA, 16), (kf.KF_AOSOA, 128)])
def test_noalloc_matches_workspace_entry_on_consecutive_calls(dev, layout, host_path):
    # Two consecutive no-allocation calls per workload, and workloads of
    # different kinds, sizes and precisions one after another: each call must
    # see only its own data in the shared staging buffer.  75,003 tracks span
    # three chunks of 32,768 with a ragged tail; the KF_ADAPTIVE batch (two
    # chunks) marks tracks for the FP64 redo pass in the staged status array.
    cases = [(W.make_p2r(3, 25001, seed=21), kf.KF_FP32),
             (W.make_p2z(75003, seed=22), kf.KF_FP32),
             (_grazing_p2r(), kf.KF_ADAPTIVE),
             (W.make_p2r(1, 1000, seed=23), kf.KF_FP32)]
    for w, precision in cases:
        hb = kf.host_upload(w, layout[0], layout[1], dev, chunk_tracks=16384)
        hb.run(precision)  # the existing entry point, with a caller-provided workspace
        torch.cuda.synchronize()
        ref = hb.download()
        if precision == kf.KF_ADAPTIVE:
            # the redo pass ran: flagged and redone tracks, no mark left
            assert not np.any(ref[2] & 0x80)
        for fill in (np.nan, -7.0):
            _assert_equal(_noalloc(hb, fill, precision), ref)


def test_noalloc_calls_leave_device_memory_unchanged(dev):
    # The copy path, ten calls in a row of three chunks each: the device's
    # free memory is the same before and after (the first calls, which load
    # the kernels and look up the staging buffer's address, come before).
    kf.kf_set_host_path(kf.KF_HOST_COPY)
    try:
        w = W.make_p2r(1, 75003, seed=26)
        hb = kf.host_upload(w, kf.KF_AOSOA, 32, dev)
        kind = kf.KF_P2R
        st_out, cv_out = torch.empty_like(hb.state_out), torch.empty_like(hb.cov_out)
        status = torch.empty_like(hb.status)

        def call(precision):
            kf.kf_propagate_update_host_noalloc(
                kind, kf.make_params(w.bz, precision), hb.layout, hb.state_in, hb.cov_in,
                st_out, cv_out, hb.charge, hb.hit, hb.hit_cov, hb.surf, 0, status)

        for precision in (kf.KF_FP32, kf.KF_ADAPTIVE):
            call(precision)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for k in range(10):
            call(kf.KF_FP32 if k % 2 == 0 else kf.KF_ADAPTIVE)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
    finally:
        kf.kf_set_host_path(kf.KF_HOST_AUTO)


def test_noalloc_rejects_chunk_above_capacity(dev):
    w = W.make_p2z(100, seed=24)
    hb = kf.host_upload(w, kf.KF_SOA, 0, dev)
    with pytest.raises(kf.KfError) as e:
        kf.kf_propagate_update_host_noalloc(
            kf.KF_P2Z, kf.make_params(w.bz), hb.layout, hb.state_in, hb.cov_in, hb.state_out,
            hb.cov_out, hb.charge, hb.hit, hb.hit_cov, hb.surf, 0, hb.status,
            chunk_tracks=kf.KF_NOALLOC_MAX_CHUNK + 1)
    assert e.value.code == kf.KF_ERR_ARG
    assert "capacity" in str(e.value)
