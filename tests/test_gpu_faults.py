"""Failure detection on the GPU without a GPU fault.

The staged kernels bound every barrier wait.  Here the compute warps' limit
is set to zero polls (kf_set_device_wait_limit), so every such wait runs out
at once -- a wait on a barrier that nothing completes in time -- while the
producer warp's own waits keep their full limit and let every bulk copy it
issued land before its CTA exits.  The call must return, the device error
word must report KF_DEVERR_TIMEOUT, the outputs must be left unwritten, and
the next launch with the default limit must give the results of a fresh run,
bit for bit, with the error word clear: the context stays usable.
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
    kf.kf_take_device_error()
    yield torch.device("cuda:0")
    kf.kf_set_device_wait_limit(-1)
    kf.kf_set_step_kernel(kf.KF_STEP_AUTO)
    kf.kf_set_staged_ctas_per_sm(0)
    assert kf.kf_take_device_error() == 0


def _workload(kind):
    # several tiles per CTA at every launch shape (76,800 tracks = 300 tiles)
    return W.make_p2z(76800, seed=31) if kind == W.P2Z else W.make_p2r(8, 9600, seed=31)


@pytest.mark.parametrize("ctas", [2, 3])
@pytest.mark.parametrize("kind", [W.P2Z, W.P2R], ids=["p2z", "p2r"])
def test_staged_step_wait_runs_out_and_the_context_recovers(dev, kind, ctas):
    w = _workload(kind)
    kf.kf_set_step_kernel(kf.KF_STEP_STAGED)
    kf.kf_set_staged_ctas_per_sm(ctas)
    try:
        fresh = kf.upload(w, kf.KF_AOSOA, 32, dev)
        fresh.run()
        torch.cuda.synchronize()
        ref = fresh.download()
        assert kf.kf_take_device_error() == 0

        b = kf.upload(w, kf.KF_AOSOA, 32, dev)
        b.state_out.fill_(float("nan"))
        b.cov_out.fill_(float("nan"))
        kf.kf_set_device_wait_limit(0)
        try:
            b.run()  # returns: the launch itself succeeds
            torch.cuda.synchronize()
        finally:
            kf.kf_set_device_wait_limit(-1)
        assert kf.kf_take_device_error() == kf.KF_DEVERR_TIMEOUT
        # every compute warp gave up at its first tile: nothing was written
        assert bool(torch.isnan(b.state_out).all()) and bool(torch.isnan(b.cov_out).all())
        assert int(b.status.count_nonzero()) == 0

        # the same buffers, default limit: a fresh run's results, bit for bit
        b.run()
        torch.cuda.synchronize()
        got = b.download()
        assert kf.kf_take_device_error() == 0
        for x, y in zip(ref, got):
            assert np.array_equal(x, y)
    finally:
        kf.kf_set_step_kernel(kf.KF_STEP_AUTO)
        kf.kf_set_staged_ctas_per_sm(0)


def test_compressed_staged_wait_runs_out_and_the_context_recovers(dev):
    w = _workload(W.P2R)
    lay = kf.make_layout(kf.KF_AOSOA, 32, w.n)
    sig, rho = W.compress_cov(w.cov)
    ins = (kf.to_device(w.state, lay, dev), kf.to_device(sig, lay, dev),
           kf.to_device_rho(rho, lay, dev))
    rest = (torch.from_numpy(w.charge).to(dev), kf.to_device(w.hit, lay, dev),
            kf.to_device(w.hitcov, lay, dev),
            torch.tensor([w.surf], dtype=torch.float32, device=dev))

    def launch(outs, status):
        kf.kf_propagate_update_compressed(kf.KF_P2R, kf.make_params(w.bz), lay, *ins, *outs,
                                          *rest, 0, status)
        torch.cuda.synchronize()

    ref = tuple(torch.empty_like(t) for t in ins)
    ref_status = torch.zeros(w.n, dtype=torch.uint8, device=dev)
    launch(ref, ref_status)
    assert kf.kf_take_device_error() == 0

    outs = tuple(torch.full_like(t, float("nan")) for t in ins)
    status = torch.zeros(w.n, dtype=torch.uint8, device=dev)
    kf.kf_set_device_wait_limit(0)
    try:
        launch(outs, status)
    finally:
        kf.kf_set_device_wait_limit(-1)
    assert kf.kf_take_device_error() == kf.KF_DEVERR_TIMEOUT
    assert all(bool(torch.isnan(t).all()) for t in outs)

    launch(outs, status)
    assert kf.kf_take_device_error() == 0
    for x, y in zip(ref, outs):
        assert torch.equal(x, y)
    assert torch.equal(ref_status, status)

