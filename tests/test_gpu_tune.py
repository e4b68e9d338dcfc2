"""The autotuner through the C ABI: it picks a valid launch shape, leaves
results unchanged bit for bit, round-trips its cache as text, and the chain
tuner leaves the caller's state as it was."""
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
    kf.kf_set_step_kernel(kf.KF_STEP_AUTO)
    kf.autotune_clear()
    yield torch.device("cuda:0")
    kf.autotune_clear()


@pytest.mark.parametrize("layout,shape", [((kf.KF_SOA, 0), (4, 9600)), ((kf.KF_SOA, 0), (1, 38401)),
                                          ((kf.KF_AOSOA, 64), (4, 9600))])
def test_step_autotune_keeps_results(dev, layout, shape):
    w = W.make_p2r(shape[0], shape[1], seed=61)
    b = kf.upload(w, layout[0], layout[1], dev)
    b.run()
    before = b.download()
    t = kf.autotune_step(b)
    assert t["step_kernel"] in ("direct", "staged") and t["ms"] > 0
    if layout[0] == kf.KF_SOA and w.n % 4:
        assert t["step_kernel"] == "direct"  # staged SoA needs n % 4 == 0
    b.status.zero_()
    b.run()  # now launched with the cached shape
    after = b.download()
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    text = kf.autotune_export()
    assert "|" in text and len(text.splitlines()) >= 1
    kf.autotune_clear()
    assert kf.autotune_export() == ""
    kf.autotune_import(text)
    assert kf.autotune_export() == text


def test_chain_autotune_leaves_state(dev):
    cw = W.make_chain(events=8, seed=62)
    dc = kf.chain_upload(cw, kf.KF_AOSOA, 32, dev)
    s0, c0 = dc.state.clone(), dc.cov.clone()
    t = kf.autotune_chain(dc)
    assert t["threads"] in (64, 128, 256)
    torch.cuda.synchronize()
    assert torch.equal(s0, dc.state) and torch.equal(c0, dc.cov)
    dc.run()
    tuned = dc.download()
    dc.reset()
    kf.autotune_clear()
    dc.run()
    plain = dc.download()
    assert np.array_equal(tuned[0], plain[0]) and np.array_equal(tuned[1], plain[1])


def test_import_rejects_malformed_text(dev):
    with pytest.raises(kf.KfError):
        kf.autotune_import("no separators here\n")
