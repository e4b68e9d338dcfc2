"""Host-side workload generation and formats (no GPU): the compressed
covariance encoding, the AoSoA layout round trip, the chain layer sequence
and event sizes, and the simulated hits lying on their surfaces."""
import numpy as np

from paper_2401_14221_gb300 import workload as W


def test_compressed_covariance_bound():
    # FP16 correlations: each element within 2^-12 of its correlation scale
    # sqrt(C_ii C_jj) (|rho| <= 1, FP16 spacing 2^-11 below 1); variances
    # within FP32 rounding of sigma^2
    w = W.make_p2r(1, 4000, seed=21, pt_range=(0.2, 100.0))
    sig, rho = W.compress_cov(w.cov)
    assert sig.dtype == np.float32 and rho.dtype == np.float16
    assert np.all(np.abs(rho.astype(np.float64)) <= 1.0)
    back = W.decompress_cov(sig, rho)
    c = w.cov.astype(np.float64)
    for i in range(6):
        for j in range(i + 1):
            k = W.tri_index(i, j)
            scale = np.sqrt(c[W.tri_index(i, i)] * c[W.tri_index(j, j)])
            err = np.abs(back[k] - c[k]) / scale
            assert err.max() <= (2.0 ** -12 if i != j else 2.0 ** -22), (i, j, err.max())


def test_aosoa_round_trip_and_padding():
    rng = np.random.default_rng(3)
    for n in (1, 31, 32, 33, 1000):
        a = rng.standard_normal((6, n)).astype(np.float32)
        for width in (16, 32, 64, 128):
            blocks = W.to_aosoa(a, width)
            assert blocks.shape == (W.aosoa_blocks(n, width), 6, width)
            assert np.array_equal(W.from_aosoa(blocks, n), a)
            # element (c, i) sits at block i // width, slot i % width
            i = n - 1
            assert blocks[i // width, 5, i % width] == a[5, i]


def test_rho_pair_layout_round_trip_and_addresses():
    # the compressed store's correlations: per block of W tracks, pair p of
    # track r at FP16 elements 2 (p W + r) and 2 (p W + r) + 1 (rho_2p low),
    # rho_14 at 14 W + r; SoA is one block of n tracks; 15 W values per block
    rng = np.random.default_rng(5)
    for n in (1, 7, 31, 32, 33, 1000):
        rho = rng.uniform(-1, 1, (15, n)).astype(np.float16)
        for width in (None, 16, 32, 64, 128):
            flat = W.rho_to_layout(rho, width)
            w = n if width is None else width
            nb = 1 if width is None else W.aosoa_blocks(n, width)
            assert flat.dtype == np.float16 and flat.shape == (nb * 15 * w,)
            assert np.array_equal(W.rho_from_layout(flat, n, width), rho)
            for i in (0, n // 2, n - 1):
                b, r = (0, i) if width is None else (i // width, i % width)
                base = b * 15 * w
                for p in range(7):
                    assert flat[base + 2 * (p * w + r)] == rho[2 * p, i]
                    assert flat[base + 2 * (p * w + r) + 1] == rho[2 * p + 1, i]
                assert flat[base + 14 * w + r] == rho[14, i]


def test_chain_layers_alternate_and_event_sizes_clip():
    kinds, pos = W.chain_layers()
    assert len(kinds) == 15 and list(kinds[:4]) == [W.P2R, W.P2Z, W.P2R, W.P2Z]
    assert np.allclose(pos[kinds == W.P2R], np.linspace(4, 110, 8))
    assert np.allclose(pos[kinds == W.P2Z], np.linspace(30, 280, 7))
    sizes = W.lognormal_event_sizes(np.random.default_rng(1), 20000)
    assert sizes.min() >= 500 and sizes.max() <= 40000
    assert abs(np.median(sizes) - 5000) < 250


def test_hits_lie_on_their_surfaces():
    w = W.make_p2r(1, 2000, seed=22)
    r = np.hypot(w.hit[0], w.hit[1])
    assert np.allclose(r[w.reached], w.surf, rtol=1e-6)
    w = W.make_p2z(2000, seed=23)
    assert np.allclose(w.hit[2][w.reached], w.surf, rtol=1e-6)
