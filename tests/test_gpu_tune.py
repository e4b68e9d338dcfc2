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


@pytest.mark.parametrize("width,n", [(128, 77777), (16, 38401), (32, 1000)])
def test_direct_cta_sizes_equal_bitwise(dev, width, n):
    # The one-thread-per-track kernel at every CTA size the tuner may pick:
    # a 64-thread CTA covers half of a 128-wide AoSoA block (its L2 prefetch
    # asks for the whole block), a 256-thread CTA sixteen 16-wide blocks, and
    # the last CTA is ragged.  The per-track arithmetic is the same, so the
    # results are bitwise equal, in place as well.
    w = W.make_p2r(1, n, seed=63)
    b = kf.upload(w, kf.KF_AOSOA, width, dev)
    kf.autotune_clear()
    kf.autotune_step(b)  # learn this GPU's cache key for the batch
    fields = kf.autotune_export().splitlines()[0].split("|")
    outs = []
    for threads in (64, 128, 256):
        fields[7], fields[8], fields[9] = str(kf.KF_STEP_DIRECT), str(threads), "0"
        kf.autotune_clear()
        kf.autotune_import("|".join(fields) + "\n")
        b.status.zero_()
        b.run()
        outs.append(b.download())
    kf.autotune_clear()
    for o in outs[1:]:
        for x, y in zip(outs[0], o):
            assert np.array_equal(x, y)
    fields[8] = "64"
    kf.autotune_import("|".join(fields) + "\n")
    b.status.zero_()
    b.run(in_place=True)
    kf.autotune_clear()
    got = (kf.from_device(b.state_in, 6, b.n, b.layout),
           kf.from_device(b.cov_in, 21, b.n, b.layout), b.status.cpu().numpy())
    for x, y in zip(outs[0], got):
        assert np.array_equal(x, y)
