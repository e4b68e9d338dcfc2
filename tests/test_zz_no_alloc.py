"""kf_propagate_update_host_noalloc against the workspace host-array entry point.

The no-allocation entry point is for callers that may not call cudaMalloc (a
plugin whose host process owns the device allocator, or a latency-critical
loop where an allocation would synchronise the device): it stages host
arrays through a fixed device buffer held by the library instead of a
caller-provided workspace.  Its results must match
kf_p2r/p2z_propagate_update_host within the parity bounds, call after call,
while every call reuses the same staging buffer.  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest
import torch

from oracle import compare
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


def _noalloc(hb, fill):
    """Run the no-allocation call on the host arrays of `hb`, writing into
    fresh host outputs pre-filled with `fill`; returns SoA results."""
    st_out = torch.full_like(hb.state_out, fill)
    cv_out = torch.full_like(hb.cov_out, fill)
    status = torch.full_like(hb.status, 255)
    kind = kf.KF_P2Z if hb.kind == W.P2Z else kf.KF_P2R
    kf.kf_propagate_update_host_noalloc(
        kind, kf.make_params(hb.bz), hb.layout, hb.state_in, hb.cov_in, st_out, cv_out,
        hb.charge, hb.hit, hb.hit_cov, hb.surf, int(hb.surf.numel() > 1), status)
    torch.cuda.synchronize()
    saved = hb.state_out, hb.cov_out, hb.status
    hb.state_out, hb.cov_out, hb.status = st_out, cv_out, status
    out = hb.download()
    hb.state_out, hb.cov_out, hb.status = saved
    return out


def _assert_match(got, ref):
    rep = compare.compare(got[0].T, got[1].T, got[2], ref[0].T, ref[1].T, ref[2])
    assert rep["ok"], rep


@pytest.mark.parametrize("layout", [(kf.KF_SOA, 0), (kf.KF_AOSOA, 16), (kf.KF_AOSOA, 128)])
def test_noalloc_matches_workspace_entry_on_consecutive_calls(dev, layout, host_path):
    # Two consecutive no-allocation calls per workload, and workloads of
    # different kinds and sizes one after another: each call must see only
    # its own data in the shared staging buffer.  75,003 tracks span three
    # chunks of 32,768 with a ragged tail.
    workloads = [W.make_p2r(3, 25001, seed=21), W.make_p2z(75003, seed=22),
                 W.make_p2r(1, 1000, seed=23)]
    for w in workloads:
        hb = kf.host_upload(w, layout[0], layout[1], dev, chunk_tracks=16384)
        hb.run()  # the existing entry point, with a caller-provided workspace
        torch.cuda.synchronize()
        ref = hb.download()
        for fill in (np.nan, -7.0):
            _assert_match(_noalloc(hb, fill), ref)


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
