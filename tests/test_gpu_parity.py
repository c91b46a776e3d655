"""GPU path (libencore_gpu through its C ABI) against the FP64 oracle.

Bars: neighbour counts bit-exact; every multiplet within 1e-5 of its order's RMS on
the FP32 path (within 3e-5 on the split-BF16 path).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2105_08722_gb300 import catalogs

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
TOL_BF16 = 3e-5     # split-bf16 tensor-core contraction


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_08722_gb300 import build
    build()
    oracle.build()
    return torch, torch.device("cuda:0")


def gpu_run(torch_dev, pos, w, orders, lmax, edges, box=0.0, allparity=False, wprim=None,
            prec=0, tuning=None):
    torch, dev = torch_dev
    from paper_2105_08722_gb300._lib import NPCF
    est = NPCF(lmax, orders, edges, box, prec, allparity)
    for k, v in (tuning or {}).items():
        est.set_tuning(k, v)
    tp = torch.from_numpy(np.ascontiguousarray(pos, np.float32)).to(dev)
    tw = torch.from_numpy(np.ascontiguousarray(w, np.float32)).to(dev)
    twp = None if wprim is None else torch.from_numpy(np.ascontiguousarray(wprim, np.float32)).to(dev)
    est.accumulate(tp, tw, wprim=twp)
    return est, est.finalize(), est.pair_counts()


def assert_orders_close(got, want, orders, lmax, nr, allparity=False, tol=TOL_FP32):
    g = oracle.split_orders(got, orders, lmax, nr, allparity)
    o = oracle.split_orders(want, orders, lmax, nr, allparity)
    for N in orders:
        rms = math.sqrt(float(np.mean(o[N] ** 2)))
        assert rms > 0
        err = float(np.max(np.abs(g[N] - o[N]))) / rms
        assert err <= tol, "order %d: max |gpu - oracle| / rms = %.3e" % (N, err)


def _catalog(n, side, seed, weights=True):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0, side, size=(n, 3)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, size=n).astype(np.float32) if weights else np.ones(n, np.float32)
    return pos, w


# ------------------------------------------------------------------ neighbour counts

@pytest.mark.parametrize("n,box,edges", [
    (1, 50.0, [0.0, 5.0, 10.0]),
    (2, 50.0, [0.0, 5.0, 10.0]),
    (33, 60.0, [1.0, 4.0, 9.0, 15.0]),
    (1000, 100.0, list(np.linspace(0.0, 30.0, 11))),
    (5003, 200.0, list(np.linspace(5.0, 50.0, 16))),
    (777, 0.0, list(np.linspace(2.0, 20.0, 7))),
])
def test_pair_counts_bit_exact(torch_dev, n, box, edges):
    pos, w = _catalog(n, box if box > 0 else 80.0, 100 + n)
    for k in (1, 3, 4):   # several cell sizes must give the same neighbour sets
        est, _, counts = gpu_run(torch_dev, pos, w, (3,), 2, edges, box, tuning={0: k})
        assert np.array_equal(counts, oracle.pair_counts(pos, edges, box)), k
        est.close()


@pytest.mark.parametrize("box", [0.0, 220.0])
def test_x_window_cut_keeps_every_neighbour(torch_dev, box):
    # the pair kernel cuts staged rows to each primary's x-window; with the cut on or off,
    # for several cell sizes, the neighbour sets (hence counts) must be the same
    pos = catalogs.lognormal_box(6000, 220.0, 32, seed=77)
    w = np.ones(len(pos), np.float32)
    edges = np.linspace(3.0, 40.0, 9)
    want = oracle.pair_counts(pos, edges, box)
    ref = None
    for k in (1, 3, 5):
        for t in (0, 1):
            _, z, counts = gpu_run(torch_dev, pos, w, (3,), 4, edges, box, tuning={0: k, 7: t})
            assert np.array_equal(counts, want), (k, t)
            if ref is None:
                ref = z
            scale = np.sqrt(np.mean(ref ** 2))
            assert np.max(np.abs(z - ref)) <= 1e-5 * scale, (k, t)


def test_pair_counts_on_exact_edges_and_duplicates(torch_dev):
    # secondaries placed at exactly representable distances equal to the shell edges,
    # coincident points and points at |d| = L/2 in a periodic box
    edges = [0.0, 2.0, 4.0, 8.0]
    base = np.array([20.0, 20.0, 20.0], np.float32)
    pts = [base, base.copy()]                                  # coincident pair
    for e in edges:
        for ax in range(3):
            p = base.copy()
            p[ax] += np.float32(e)
            pts.append(p)
            q = base.copy()
            q[ax] -= np.float32(e)
            pts.append(q)
    pts.append(np.array([0.0, 20.0, 20.0], np.float32))
    pts.append(np.array([39.5, 20.0, 20.0], np.float32))        # 0.5 apart through the wall
    pos = np.array(pts, np.float32)
    w = np.ones(len(pos), np.float32)
    for box in (0.0, 40.0):
        _, _, counts = gpu_run(torch_dev, pos, w, (3,), 1, edges, box)
        assert np.array_equal(counts, oracle.pair_counts(pos, edges, box)), box


def test_zero_and_negative_weights_counts_and_zeta(torch_dev):
    # Algorithm 1 visits every primary and every secondary within the shells: a primary of
    # weight 0 adds nothing to zeta but its pairs are still counted. About 10 % of the
    # weights are exactly 0 and the signs are mixed (as in data-minus-randoms catalogs).
    rng = np.random.default_rng(4242)
    n, box = 3000, 120.0
    pos = rng.uniform(0, box, size=(n, 3)).astype(np.float32)
    w = rng.uniform(-1.5, 1.5, size=n).astype(np.float32)
    w[rng.random(n) < 0.1] = 0.0
    assert (w == 0).sum() > 200 and (w < 0).sum() > 1000
    edges = np.linspace(4.0, 30.0, 7)
    for prec, tol in ((0, TOL_FP32), (1, TOL_BF16)):
        est, got, counts = gpu_run(torch_dev, pos, w, (3, 4), 3, edges, box, prec=prec)
        assert np.array_equal(counts, oracle.pair_counts(pos, edges, box)), prec
        want, wc = oracle.npcf(pos, w, (3, 4), 3, edges, box)
        assert np.array_equal(counts, wc)
        assert_orders_close(got, want, (3, 4), 3, len(edges) - 1, tol=tol)
        est.close()


# ------------------------------------------------------------------ a_lm

@pytest.mark.parametrize("lmax", [6, 8, 10])
def test_alm_of_sampled_primaries(torch_dev, lmax):
    pos, w = _catalog(4000, 150.0, 7)
    edges = np.linspace(5.0, 40.0, 8)
    est, _, _ = gpu_run(torch_dev, pos, w, (3,), lmax, edges, 150.0)
    sample = np.array([0, 1, 17, 500, 1999, 3998, 3999])
    a_gpu, c_gpu = est.debug_alm(sample)
    a_orc, c_orc = oracle.alm(pos, w, sample, lmax, edges, 150.0)
    assert np.array_equal(c_gpu, c_orc)
    for l in range(lmax + 1):
        for m in range(l + 1):
            g = a_gpu[:, :, l * (l + 1) // 2 + m]
            o = a_orc[:, :, l * l + l + m]
            scale = np.sqrt(np.mean(np.abs(a_orc) ** 2))
            assert np.max(np.abs(g - o)) <= 1e-5 * scale, (l, m)


# ------------------------------------------------------------------ multiplets

def test_3pcf_uniform_4096_box250_full(torch_dev):
    wl = catalogs.uniform4k_3pcf()
    _, got, counts = gpu_run(torch_dev, wl.pos, wl.w, wl.orders, wl.lmax, wl.edges, wl.box)
    want, wcounts = oracle.npcf(wl.pos, wl.w, wl.orders, wl.lmax, wl.edges, wl.box)
    assert np.array_equal(counts, wcounts)
    assert_orders_close(got, want, wl.orders, wl.lmax, len(wl.edges) - 1)


@pytest.mark.parametrize("highl", [0, 1])
@pytest.mark.parametrize("nr,lmax,n", [(3, 4, 1500), (13, 3, 2100), (16, 2, 901)])
def test_4pcf_shell_counts_and_ragged_tiles(torch_dev, nr, lmax, n, highl):
    # the FP32 contractions specialise on the number of shells after b1 and take
    # primaries in tiles of 64 (staged coupling terms) or 32 (the high-lmax kernel, forced
    # by tuning key 4): few and many shells, n not a multiple of either tile
    pos, w = _catalog(n, 160.0, 900 + nr)
    edges = np.linspace(4.0, 40.0, nr + 1)
    _, got, _ = gpu_run(torch_dev, pos, w, (4,), lmax, edges, 160.0, allparity=True,
                        tuning={4: highl})
    want, _ = oracle.npcf(pos, w, (4,), lmax, edges, 160.0, allparity=True)
    assert_orders_close(got, want, (4,), lmax, nr, allparity=True)


@pytest.mark.parametrize("highl", [0, 1])
def test_4pcf_3pcf_periodic_lmax5_10_shells(torch_dev, highl):
    pos = catalogs.lognormal_box(2500, 300.0, 64, seed=31)
    w = np.ones(len(pos), np.float32)
    edges = np.linspace(8.0, 60.0, 11)
    _, got, counts = gpu_run(torch_dev, pos, w, (3, 4), 5, edges, 300.0, tuning={4: highl})
    want, wcounts = oracle.npcf(pos, w, (3, 4), 5, edges, 300.0)
    assert np.array_equal(counts, wcounts)
    assert_orders_close(got, want, (3, 4), 5, 10)


@pytest.mark.parametrize("lmax", [6, 8, 10])
def test_high_lmax_3pcf_and_4pcf_or_refusal(torch_dev, lmax):
    # the paper's lmax = 10 setting on a small catalog. The 3PCF takes any lmax <= 10; the
    # FP32 4PCF stages the coupling terms and a tile of a_lm up to lmax 6 and switches to
    # the high-lmax kernel (terms through L1) beyond; the split-bf16 one stages them and
    # one 128-row operand slab per m3 in shared memory and is refused at create (or
    # accumulate) where those exceed it, beyond lmax 5
    from paper_2105_08722_gb300._lib import NPCFError
    pos = catalogs.lognormal_box(400, 100.0, 32, seed=81)
    w = np.ones(len(pos), np.float32)
    edges = np.linspace(5.0, 30.0, 5)
    want, wcounts = oracle.npcf(pos, w, (3, 4), lmax, edges, 100.0)
    want3, _ = oracle.npcf(pos, w, (3,), lmax, edges, 100.0)
    _, got3, counts = gpu_run(torch_dev, pos, w, (3,), lmax, edges, 100.0)
    assert np.array_equal(counts, wcounts)
    assert_orders_close(got3, want3, (3,), lmax, 4)
    for prec, tol, lmax_ok in ((0, TOL_FP32, 10), (1, TOL_BF16, 5)):
        try:
            _, got, _ = gpu_run(torch_dev, pos, w, (3, 4), lmax, edges, 100.0, prec=prec)
        except NPCFError as e:
            assert lmax > lmax_ok and "memory" in str(e), str(e)
        else:
            assert_orders_close(got, want, (3, 4), lmax, 4, tol=tol)


@pytest.mark.parametrize("lmax,nr,n", [(10, 16, 700), (10, 10, 333), (0, 2, 97)])
def test_3pcf_tiles_of_32_16_primaries_and_few_shells(torch_dev, lmax, nr, n):
    # the 3PCF stages tiles of 32 primaries where they fit in shared memory and of 16
    # beyond (lmax 10 with 16 shells: 11 x 120 outputs); n is not a multiple of a tile
    pos, w = _catalog(n, 150.0, 1100 + nr)
    edges = np.linspace(3.0, 45.0, nr + 1)
    _, got, counts = gpu_run(torch_dev, pos, w, (3,), lmax, edges, 0.0)
    want, wcounts = oracle.npcf(pos, w, (3,), lmax, edges, 0.0)
    assert np.array_equal(counts, wcounts)
    assert_orders_close(got, want, (3,), lmax, nr)


def test_4pcf_lmax10_10_shells_paper_setting(torch_dev):
    # Table 2's 4PCF at lmax = 10 with N_r = 10 shells (the high-lmax kernel), on a small
    # periodic log-normal catalog against the oracle; and lmax 7 all-parity with 16 shells
    pos = catalogs.lognormal_box(400, 250.0, 32, seed=83)
    w = np.ones(len(pos), np.float32)
    edges = np.linspace(10.0, 80.0, 11)
    _, got, counts = gpu_run(torch_dev, pos, w, (3, 4), 10, edges, 250.0)
    want, wcounts = oracle.npcf(pos, w, (3, 4), 10, edges, 250.0)
    assert np.array_equal(counts, wcounts)
    assert_orders_close(got, want, (3, 4), 10, 10)
    pos, w = _catalog(300, 120.0, 84)
    edges = np.linspace(5.0, 45.0, 17)
    _, got, _ = gpu_run(torch_dev, pos, w, (4,), 7, edges, 0.0, allparity=True)
    want, _ = oracle.npcf(pos, w, (4,), 7, edges, 0.0, allparity=True)
    assert_orders_close(got, want, (4,), 7, 16, allparity=True)


@pytest.mark.parametrize("highl", [0, 1])
def test_4pcf_all_parity_non_periodic_weighted(torch_dev, highl):
    pos, w = _catalog(1500, 120.0, 41)
    w = w - np.float32(0.9)          # mixed-sign weights, like data minus randoms
    edges = np.linspace(6.0, 36.0, 7)
    _, got, counts = gpu_run(torch_dev, pos, w, (3, 4), 4, edges, 0.0, allparity=True,
                             tuning={4: highl})
    want, wcounts = oracle.npcf(pos, w, (3, 4), 4, edges, 0.0, allparity=True)
    assert np.array_equal(counts, wcounts)
    assert_orders_close(got, want, (3, 4), 4, 6, allparity=True)


def test_lmax0_single_shell_and_tiny_catalogs(torch_dev):
    for n in (0, 1, 5):
        pos, w = _catalog(max(n, 1), 30.0, 50 + n)
        pos, w = pos[:n], w[:n]
        edges = [1.0, 12.0]
        if n == 0:
            from paper_2105_08722_gb300._lib import NPCF
            est = NPCF(0, (3,), edges, 0.0)
            assert np.all(est.finalize() == 0)
            continue
        _, got, counts = gpu_run(torch_dev, pos, w, (3,), 0, edges, 0.0)
        want, wcounts = oracle.npcf(pos, w, (3,), 0, edges, 0.0)
        assert np.array_equal(counts, wcounts)
        assert got.shape == want.shape and np.all(got == 0) and np.all(want == 0)


@pytest.mark.parametrize("tuning", [
    {},                 # every bucket summed once per primary
    {3: 2048},          # buckets that fill and are summed during the scan
    {5: 1},             # one primary per chunk
    {5: 1000, 3: 2048}, # chunks larger than a block's share, buckets summed during the scan
    {7: 0},             # whole rows, no x-window cut
    {0: 1},             # one cell per r_max: long rows
])
def test_dense_primaries_tuning_variants(torch_dev, tuning):
    # ~1000 neighbours per primary: with 2048 bucket entries per warp (512 per shell) the
    # buckets of the outer shells are summed during the scan
    pos, w = _catalog(9000, 60.0, 61)
    edges = np.linspace(2.0, 18.0, 5)
    _, got, counts = gpu_run(torch_dev, pos, w, (3, 4), 3, edges, 60.0, tuning=tuning)
    want, wcounts = oracle.npcf(pos, w, (3, 4), 3, edges, 60.0)
    assert np.array_equal(counts, wcounts)
    assert_orders_close(got, want, (3, 4), 3, 4)


@pytest.mark.parametrize("edges", [
    list(np.linspace(20.0, 160.0, 11)),           # the bench's shells: table on
    [0.0, 2.0, 4.0, 8.0],                        # r_min = 0: the r2 > 0 change and edge 0 share bin 0
    list(np.geomspace(0.02, 40.0, 17)),          # tiny inner shells: no table fits, computed shell
])
def test_shell_table_and_computed_shell_agree(torch_dev, edges):
    # the pair kernel reads a candidate's shell from a table over bins of r2 when every
    # bin holds at most one shell change (tuning key 8 = 1), else computes it; both apply
    # the same exact FP32 rule, so the counts are the oracle's in both settings
    box = 3.2 * edges[-1] + 1.0
    pos = catalogs.lognormal_box(6000, box, 32, seed=81)
    # points at exactly representable distances of 2, 4, 8 from a base point
    base = np.array([box / 2, box / 2, box / 2], np.float32)
    extra = [base]
    for e in (2.0, 4.0, 8.0):
        for ax in range(3):
            p_ = base.copy(); p_[ax] += np.float32(e); extra.append(p_)
    pos = np.concatenate([pos, np.array(extra, np.float32)])
    w = np.ones(len(pos), np.float32)
    want = oracle.pair_counts(pos, edges, box)
    ref = None
    for key8 in (1, 0):
        _, z, counts = gpu_run(torch_dev, pos, w, (3,), 3, edges, box, tuning={8: key8})
        assert np.array_equal(counts, want), key8
        if ref is None:
            ref = z
        assert np.max(np.abs(z - ref)) <= 1e-5 * np.sqrt(np.mean(ref ** 2)), key8


def test_sixteen_shells_minimum_buckets(torch_dev):
    # 16 shells and 8192 bucket entries per warp: every shell's bucket holds the minimum
    # of 512 entries, so the outer buckets are summed during the scan
    pos, w = _catalog(6000, 70.0, 63)
    edges = np.linspace(1.0, 20.0, 17)
    want, wcounts = oracle.npcf(pos, w, (3,), 4, edges, 70.0)
    for tuning in ({}, {3: 8192}):
        _, got, counts = gpu_run(torch_dev, pos, w, (3,), 4, edges, 70.0, tuning=tuning)
        assert np.array_equal(counts, wcounts), tuning
        assert_orders_close(got, want, (3,), 4, 16)


def test_non_periodic_signed_weights(torch_dev):
    # data-minus-randoms style weights in an open box (rows cut at the box faces), with the
    # default chunks and with chunks of 3 primaries
    pos, w = _catalog(4000, 60.0, 62)
    w = np.where(np.arange(len(w)) % 4 == 0, np.float32(-0.25), w).astype(np.float32)
    edges = np.linspace(3.0, 15.0, 5)
    want, wcounts = oracle.npcf(pos, w, (3, 4), 3, edges, 0.0)
    for tuning in ({}, {5: 3}):
        _, got, counts = gpu_run(torch_dev, pos, w, (3, 4), 3, edges, 0.0, tuning=tuning)
        assert np.array_equal(counts, wcounts), tuning
        assert_orders_close(got, want, (3, 4), 3, 4)


def test_accumulate_coadds_and_reset(torch_dev):
    torch, dev = torch_dev
    from paper_2105_08722_gb300._lib import NPCF
    a_pos, a_w = _catalog(800, 100.0, 71)
    b_pos, b_w = _catalog(900, 100.0, 72)
    edges = np.linspace(4.0, 30.0, 6)
    est = NPCF(3, (3, 4), edges, 100.0)
    for p, ww in ((a_pos, a_w), (b_pos, b_w)):
        est.accumulate(torch.from_numpy(p).to(dev), torch.from_numpy(ww).to(dev))
    got = est.finalize()
    za, _ = oracle.npcf(a_pos, a_w, (3, 4), 3, edges, 100.0)
    zb, _ = oracle.npcf(b_pos, b_w, (3, 4), 3, edges, 100.0)
    assert_orders_close(got, za + zb, (3, 4), 3, 5)
    est.reset()
    assert np.all(est.finalize() == 0) and np.all(est.pair_counts() == 0)


def test_host_entry_point_matches_device_entry_point(torch_dev):
    from paper_2105_08722_gb300._lib import NPCF
    pos, w = _catalog(1200, 90.0, 81)
    edges = np.linspace(3.0, 25.0, 6)
    _, dev_out, dev_counts = gpu_run(torch_dev, pos, w, (3, 4), 4, edges, 90.0)
    est = NPCF(4, (3, 4), edges, 90.0)
    est.accumulate_host(pos, w)
    assert np.array_equal(est.finalize(), dev_out)
    assert np.array_equal(est.pair_counts(), dev_counts)


def test_primary_weights_select_a_sample(torch_dev):
    pos, w = _catalog(2000, 120.0, 91)
    edges = np.linspace(4.0, 30.0, 7)
    rng = np.random.default_rng(92)
    sample = np.sort(rng.choice(len(pos), 50, replace=False))
    wp = np.zeros(len(pos), np.float32)
    wp[sample] = w[sample]
    _, got, _ = gpu_run(torch_dev, pos, w, (3, 4), 4, edges, 120.0, wprim=wp)
    want, _ = oracle.npcf(pos, w, (3, 4), 4, edges, 120.0, prim=sample)
    assert_orders_close(got, want, (3, 4), 4, 6)


def test_periodic_normalisation(torch_dev):
    pos, w = _catalog(1500, 100.0, 95, weights=False)
    edges = np.linspace(5.0, 30.0, 6)
    est, raw, _ = gpu_run(torch_dev, pos, w, (3, 4), 2, edges, 100.0)
    norm = est.finalize(normalize=True)
    V = 100.0 ** 3
    nbar = len(pos) / V
    vb = 4 * math.pi / 3 * (edges[1:] ** 3 - edges[:-1] ** 3)
    parts_raw = est.split(raw)
    parts = est.split(norm)
    for N in (3, 4):
        _, bins = est.layout(N)
        vB = V * np.prod(vb[bins], axis=1)
        R0 = (4 * math.pi) ** (-(N - 1) / 2) * nbar ** N
        assert np.allclose(parts[N], parts_raw[N] / (vB * R0), rtol=1e-12)


# ------------------------------------------------------------------ full-size workload

@pytest.fixture(scope="module")
def lognormal_workload():
    return catalogs.lognormal200k_4pcf()


def test_lognormal_200k_4pcf_sampled_primaries(torch_dev, lognormal_workload):
    """The 200k log-normal 4PCF+3PCF workload at full size, in the bench's launch
    configuration; the oracle evaluates a seeded sample of primaries one by one."""
    wl = lognormal_workload
    rng = np.random.default_rng(2024)
    sample = np.sort(rng.choice(wl.n, 48, replace=False))
    wp = np.zeros(wl.n, np.float32)
    wp[sample] = wl.w[sample]
    est, got, _ = gpu_run(torch_dev, wl.pos, wl.w, wl.orders, wl.lmax, wl.edges, wl.box, wprim=wp)
    a_gpu, c_gpu = est.debug_alm(sample)
    a_orc, c_orc = oracle.alm(wl.pos, wl.w, sample, wl.lmax, wl.edges, wl.box)
    assert np.array_equal(c_gpu, c_orc)
    want, _ = oracle.npcf(wl.pos, wl.w, wl.orders, wl.lmax, wl.edges, wl.box, prim=sample)
    assert_orders_close(got, want, wl.orders, wl.lmax, len(wl.edges) - 1)


def test_lognormal_200k_full_run_is_sum_of_complementary_samples(torch_dev, lognormal_workload):
    wl = lognormal_workload
    _, full, cfull = gpu_run(torch_dev, wl.pos, wl.w, wl.orders, wl.lmax, wl.edges, wl.box)
    mask = (np.arange(wl.n) % 3 == 0).astype(np.float32)
    _, a, ca = gpu_run(torch_dev, wl.pos, wl.w, wl.orders, wl.lmax, wl.edges, wl.box, wprim=wl.w * mask)
    _, b, cb = gpu_run(torch_dev, wl.pos, wl.w, wl.orders, wl.lmax, wl.edges, wl.box,
                       wprim=wl.w * (1 - mask))
    assert np.array_equal(ca + cb, cfull)
    # the two runs sum different primary subsets in FP32 within each chunk
    assert_orders_close(a + b, full, wl.orders, wl.lmax, len(wl.edges) - 1)


# ------------------------------------------------------------------ split-bf16 tensor-core contraction

def test_4pcf_split_bf16_periodic_lmax5_10_shells(torch_dev):
    pos = catalogs.lognormal_box(2500, 300.0, 64, seed=31)
    w = np.ones(len(pos), np.float32)
    edges = np.linspace(8.0, 60.0, 11)
    _, got, counts = gpu_run(torch_dev, pos, w, (3, 4), 5, edges, 300.0, prec=1)
    want, wcounts = oracle.npcf(pos, w, (3, 4), 5, edges, 300.0)
    assert np.array_equal(counts, wcounts)
    assert_orders_close(got, want, (3, 4), 5, 10, tol=TOL_BF16)


def test_4pcf_split_bf16_all_parity_weighted(torch_dev):
    pos, w = _catalog(1500, 120.0, 41)
    w = w - np.float32(0.9)
    edges = np.linspace(6.0, 36.0, 7)
    _, got, counts = gpu_run(torch_dev, pos, w, (3, 4), 4, edges, 0.0, allparity=True, prec=1)
    want, wcounts = oracle.npcf(pos, w, (3, 4), 4, edges, 0.0, allparity=True)
    assert np.array_equal(counts, wcounts)
    assert_orders_close(got, want, (3, 4), 4, 6, allparity=True, tol=TOL_BF16)


def test_split_bf16_and_fp32_paths_agree_on_ragged_chunks(torch_dev):
    # chunk sizes that leave partial steps of 16 primaries and empty blocks
    pos, w = _catalog(1037, 100.0, 43)
    edges = np.linspace(4.0, 30.0, 9)
    for chunk in (1, 15, 17, 1000, 5000):
        _, a, _ = gpu_run(torch_dev, pos, w, (4,), 3, edges, 100.0, prec=1, tuning={2: chunk})
        _, b, _ = gpu_run(torch_dev, pos, w, (4,), 3, edges, 100.0, prec=0, tuning={2: chunk})
        assert_orders_close(a, b, (4,), 3, 8, tol=TOL_BF16)


def test_lognormal_200k_split_bf16_sampled_primaries(torch_dev, lognormal_workload):
    wl = lognormal_workload
    rng = np.random.default_rng(2025)
    sample = np.sort(rng.choice(wl.n, 48, replace=False))
    wp = np.zeros(wl.n, np.float32)
    wp[sample] = wl.w[sample]
    _, got, _ = gpu_run(torch_dev, wl.pos, wl.w, wl.orders, wl.lmax, wl.edges, wl.box, wprim=wp, prec=1)
    want, _ = oracle.npcf(wl.pos, wl.w, wl.orders, wl.lmax, wl.edges, wl.box, prim=sample)
    assert_orders_close(got, want, wl.orders, wl.lmax, len(wl.edges) - 1, tol=TOL_BF16)


# ------------------------------------------------------------------ 5PCF

# tuning key 9: 0 = automatic, 1 = the register-only kernel, 2 = P34 cached in shared
# memory per block with the coupling terms read through L1, 3 = the same with the terms in
# shared memory too; every kernel runs on the same cases
@pytest.mark.parametrize("regonly", [0, 1, 2, 3])
def test_5pcf_periodic_lmax3(torch_dev, regonly):
    pos = catalogs.lognormal_box(900, 150.0, 32, seed=51)
    w = np.ones(len(pos), np.float32)
    edges = np.linspace(6.0, 42.0, 7)
    _, got, counts = gpu_run(torch_dev, pos, w, (5,), 3, edges, 150.0, tuning={9: regonly})
    want, wcounts = oracle.npcf(pos, w, (5,), 3, edges, 150.0)
    assert np.array_equal(counts, wcounts)
    assert_orders_close(got, want, (5,), 3, 6)


@pytest.mark.parametrize("regonly", [0, 1, 2, 3])
@pytest.mark.parametrize("nr", [4, 9, 10])
def test_5pcf_many_shells(torch_dev, nr, regonly):
    # 4 shells: one bin tuple; 9 and 10 shells take items of 1 to 4 multiplets sharing
    # (l12 l3 l4), by b2, and the widest P34 caches
    pos = catalogs.lognormal_box(700, 150.0, 32, seed=53)
    w = np.ones(len(pos), np.float32)
    edges = np.linspace(4.0, 40.0, nr + 1)
    _, got, counts = gpu_run(torch_dev, pos, w, (5,), 3, edges, 150.0, tuning={9: regonly})
    want, wcounts = oracle.npcf(pos, w, (5,), 3, edges, 150.0)
    assert np.array_equal(counts, wcounts)
    assert_orders_close(got, want, (5,), 3, nr)


@pytest.mark.parametrize("regonly", [0, 1, 2, 3])
def test_5pcf_lmax5_10_shells(torch_dev, regonly):
    # the paper's 5PCF timing setting (lmax 5, 10 shells) on a small catalog: 1,406
    # multiplets x 210 bin tuples
    pos = catalogs.lognormal_box(300, 150.0, 32, seed=91)
    w = np.ones(len(pos), np.float32)
    edges = np.linspace(4.0, 40.0, 11)
    _, got, counts = gpu_run(torch_dev, pos, w, (5,), 5, edges, 150.0, tuning={9: regonly})
    want, wcounts = oracle.npcf(pos, w, (5,), 5, edges, 150.0)
    assert np.array_equal(counts, wcounts)
    assert_orders_close(got, want, (5,), 5, 10)


@pytest.mark.parametrize("regonly", [0, 1, 2, 3])
def test_5pcf_all_parity_non_periodic_weighted_with_lower_orders(torch_dev, regonly):
    pos, w = _catalog(500, 80.0, 52)
    w = w - np.float32(0.8)
    edges = np.linspace(5.0, 30.0, 6)
    _, got, counts = gpu_run(torch_dev, pos, w, (3, 4, 5), 2, edges, 0.0, allparity=True,
                             tuning={9: regonly})
    want, wcounts = oracle.npcf(pos, w, (3, 4, 5), 2, edges, 0.0, allparity=True)
    assert np.array_equal(counts, wcounts)
    assert_orders_close(got, want, (3, 4, 5), 2, 5, allparity=True)


# ------------------------------------------------------------------ random splits, data harmonics kept

@pytest.mark.parametrize("box", [150.0, 0.0])
def test_split_with_cached_data_matches_uncached_and_oracle(torch_dev, box):
    # Sec. 4.2: the data's a_lm contributions are the same in every data-minus-randoms
    # split; npcf_cache_data forms them once and npcf_accumulate_split adds only what the
    # randoms change. Two co-added splits must equal two plain accumulate calls on the
    # concatenated catalogs (counts exactly) and the oracle.
    torch, dev = torch_dev
    from paper_2105_08722_gb300._lib import NPCF
    rng = np.random.default_rng(700)
    data = catalogs.lognormal_box(1200, 150.0, 32, seed=71)
    if box == 0.0:   # randoms reach beyond the data's bounding box in an open geometry
        r1 = rng.uniform(-10.0, 160.0, size=(1800, 3)).astype(np.float32)
        r2 = rng.uniform(-10.0, 160.0, size=(1500, 3)).astype(np.float32)
    else:
        r1 = rng.uniform(0.0, 150.0, size=(1800, 3)).astype(np.float32)
        r2 = rng.uniform(0.0, 150.0, size=(1500, 3)).astype(np.float32)
    wd = np.ones(len(data), np.float32)
    w1 = np.full(len(r1), -len(data) / len(r1), np.float32)
    w2 = np.full(len(r2), -len(data) / len(r2), np.float32)
    edges = np.linspace(5.0, 35.0, 6)
    orders, lmax = (3, 4, 5), 2
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    plain = NPCF(lmax, orders, edges, box)
    cached = NPCF(lmax, orders, edges, box)
    cached.cache_data(t(data), t(wd))
    want = 0.0
    wcounts = 0
    for r, wr in ((r1, w1), (r2, w2)):
        pos = np.concatenate([data, r])
        w = np.concatenate([wd, wr])
        plain.accumulate(t(pos), t(w))
        cached.accumulate_split(t(r), t(wr))
        z, c = oracle.npcf(pos, w, orders, lmax, edges, box)
        want = want + z
        wcounts = wcounts + c
    got, ref = cached.finalize(), plain.finalize()
    assert np.array_equal(cached.pair_counts(), plain.pair_counts())
    assert np.array_equal(cached.pair_counts(), wcounts)
    assert_orders_close(got, ref, orders, lmax, len(edges) - 1)
    assert_orders_close(got, want, orders, lmax, len(edges) - 1)
    # a split without randoms adds the data alone
    solo = NPCF(lmax, orders, edges, box)
    solo.cache_data(t(data), t(wd))
    solo.accumulate_split(t(np.zeros((0, 3), np.float32)), t(np.zeros(0, np.float32)))
    zd, cd = oracle.npcf(data, wd, orders, lmax, edges, box)
    assert np.array_equal(solo.pair_counts(), cd)
    assert_orders_close(solo.finalize(), zd, orders, lmax, len(edges) - 1)
    for e in (plain, cached, solo):
        e.close()


def test_split_needs_cached_data(torch_dev):
    torch, dev = torch_dev
    from paper_2105_08722_gb300._lib import NPCF, NPCFError, NPCF_EINVAL
    est = NPCF(2, (3,), np.linspace(5.0, 35.0, 6), 150.0)
    with pytest.raises(NPCFError) as e:
        est.accumulate_split(torch.zeros((10, 3), device=dev), torch.zeros(10, device=dev))
    assert e.value.status == NPCF_EINVAL
    est.close()


# ------------------------------------------------------------------ gridded fields (FFT)

def _mesh_centres(n, box):
    h = box / n
    c = (np.arange(n, dtype=np.float64) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")   # cells x fastest, then y, z
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float32)


@pytest.mark.parametrize("orders,lmax,allparity", [((3, 4), 3, False), ((5,), 2, True)])
def test_grid_fft_matches_oracle_on_cell_centres(torch_dev, orders, lmax, allparity):
    # Eq. (alm-binned-def-fft): the a_lm of every cell by FFT, then the usual contraction
    # with the cells as primaries of weight delta. Its plain definition is the particle
    # estimator on the cell centres with weights delta; with a power-of-two cell side the
    # centres and their differences are exact in FP32, so the shells agree exactly.
    torch, dev = torch_dev
    from paper_2105_08722_gb300._lib import NPCF
    n, box = 16, 128.0
    delta = np.random.default_rng(808).normal(size=(n, n, n)).astype(np.float32)
    edges = np.array([6.0, 13.0, 21.0, 29.0, 37.0])
    est = NPCF(lmax, orders, edges, box, allparity=allparity)
    est.accumulate_grid(torch.from_numpy(delta).to(dev))
    got = est.finalize()
    pos = _mesh_centres(n, box)
    want, _ = oracle.npcf(pos, delta.ravel(), orders, lmax, edges, box, allparity=allparity)
    assert_orders_close(got, want, orders, lmax, len(edges) - 1, allparity=allparity)
    # the particle path on the same cell centres agrees too, and a second call co-adds
    _, zp, _ = gpu_run(torch_dev, pos, delta.ravel(), orders, lmax, edges, box, allparity=allparity)
    assert_orders_close(got, zp, orders, lmax, len(edges) - 1, allparity=allparity)
    est.accumulate_grid(torch.from_numpy(delta).to(dev))
    assert_orders_close(est.finalize(), 2 * want, orders, lmax, len(edges) - 1, allparity=allparity)
    est.close()


def test_grid_fft_needs_a_periodic_box(torch_dev):
    torch, dev = torch_dev
    from paper_2105_08722_gb300._lib import NPCF, NPCFError, NPCF_EUNSUPPORTED
    est = NPCF(2, (3,), np.array([6.0, 13.0, 21.0]), 0.0)
    with pytest.raises(NPCFError) as e:
        est.accumulate_grid(torch.zeros((8, 8, 8), device=dev))
    assert e.value.status == NPCF_EUNSUPPORTED
    est.close()


# ------------------------------------------------------------------ 6PCF

@pytest.mark.parametrize("n,lmax,nr,allparity", [
    (400, 2, 8, False),   # 327 multiplets x 56 bin tuples
    (300, 3, 6, False),   # 2,212 multiplets (intermediates up to 2 lmax) x 6 bin tuples
    (400, 1, 8, True),    # all parities: 42 multiplets, parity-odd ones imaginary
    (300, 2, 5, False),   # one bin tuple
    (300, 2, 7, True),
])
def test_6pcf_periodic(torch_dev, n, lmax, nr, allparity):
    # Eq. (basis-coupling) with two intermediates, contracted through m12 and m123 on the
    # GPU; the oracle sums the full M range of Eq. (NPCF-mult-discrete-binned-estimator)
    pos = catalogs.lognormal_box(n, 150.0, 32, seed=60 + nr)
    w = np.ones(len(pos), np.float32)
    edges = np.linspace(6.0, 42.0, nr + 1)
    _, got, counts = gpu_run(torch_dev, pos, w, (6,), lmax, edges, 150.0, allparity=allparity)
    want, wcounts = oracle.npcf(pos, w, (6,), lmax, edges, 150.0, allparity=allparity)
    assert np.array_equal(counts, wcounts)
    assert_orders_close(got, want, (6,), lmax, nr, allparity=allparity)


def test_6pcf_with_lower_orders_weighted_open_box(torch_dev):
    # orders 3 to 6 in one context (output offsets), signed weights, no periodicity
    pos, w = _catalog(350, 80.0, 66)
    w = w - np.float32(0.8)
    edges = np.linspace(5.0, 30.0, 7)
    _, got, counts = gpu_run(torch_dev, pos, w, (3, 4, 5, 6), 2, edges, 0.0)
    want, wcounts = oracle.npcf(pos, w, (3, 4, 5, 6), 2, edges, 0.0)
    assert np.array_equal(counts, wcounts)
    assert_orders_close(got, want, (3, 4, 5, 6), 2, 6)


def test_6pcf_limits(torch_dev):
    from paper_2105_08722_gb300._lib import NPCF, NPCFError, NPCF_EUNSUPPORTED
    with pytest.raises(NPCFError) as e:
        NPCF(2, (6,), np.linspace(1.0, 10.0, 10), 100.0)   # 9 shells: the contraction takes 8
    assert e.value.status == NPCF_EUNSUPPORTED
    # fewer than 5 shells: no bin tuple, nothing to compute, an empty order
    est = NPCF(2, (3, 6), np.linspace(1.0, 10.0, 5), 100.0)
    assert est.layout(6)[1].shape[0] == 0
    est.close()


def test_lognormal_100k_5pcf_lmax4_sampled_primaries(torch_dev):
    wl = catalogs.lognormal100k_5pcf()
    rng = np.random.default_rng(2026)
    sample = np.sort(rng.choice(wl.n, 16, replace=False))
    wp = np.zeros(wl.n, np.float32)
    wp[sample] = wl.w[sample]
    _, got, _ = gpu_run(torch_dev, wl.pos, wl.w, wl.orders, wl.lmax, wl.edges, wl.box, wprim=wp)
    want, _ = oracle.npcf(wl.pos, wl.w, wl.orders, wl.lmax, wl.edges, wl.box, prim=sample)
    assert_orders_close(got, want, wl.orders, wl.lmax, len(wl.edges) - 1)


# ------------------------------------------------------------------ edge correction (a7)

def _ball_catalogs(seed, n_data=900, n_rand=3600, radius=55.0):
    """Data clustered inside a ball, uniform randoms in the same ball (non-periodic)."""
    rng = np.random.default_rng(seed)
    centre = np.array([60.0, 60.0, 60.0])

    def in_ball(p):
        return np.sum((p - centre) ** 2, axis=1) < radius ** 2

    r = rng.uniform(centre - radius, centre + radius, size=(4 * n_rand, 3))
    r = r[in_ball(r)][:n_rand]
    d = catalogs.lognormal_box(4 * n_data, 120.0, 32, seed=seed).astype(np.float64)
    d = d[in_ball(d)][:n_data]
    ratio = len(d) / len(r)
    pos = np.concatenate([d, r]).astype(np.float32)
    w = np.concatenate([np.ones(len(d)), np.full(len(r), -ratio)]).astype(np.float32)
    return pos, w, r.astype(np.float32), np.full(len(r), ratio, np.float32)


def _edge_contexts(torch_dev, pos, w, rpos, rw, lmax, edges):
    nctx, nraw, _ = gpu_run(torch_dev, pos, w, (3, 4), lmax, edges, 0.0)
    rctx, rraw, _ = gpu_run(torch_dev, rpos, rw, (3, 4), lmax, edges, 0.0)
    return nctx, rctx, nraw, rraw


def test_edge_correction_solve_matches_oracle_on_the_same_raw_multiplets(torch_dev):
    # the FP64 solve alone: the oracle corrects the GPU's own raw N and R
    pos, w, rpos, rw = _ball_catalogs(71)
    lmax, edges = 3, np.linspace(5.0, 30.0, 6)
    nr = len(edges) - 1
    nctx, rctx, nraw, rraw = _edge_contexts(torch_dev, pos, w, rpos, rw, lmax, edges)
    got = oracle.split_orders(nctx.edge_correct(rctx), (3, 4), lmax, nr)
    n = oracle.split_orders(nraw, (3, 4), lmax, nr)
    r = oracle.split_orders(rraw, (3, 4), lmax, nr)
    for N in (3, 4):
        want = oracle.edge_correct(N, lmax, nr, n[N], r[N])
        scale = np.sqrt(np.mean(want ** 2))
        assert np.max(np.abs(got[N] - want)) <= 1e-10 * scale, N


def test_edge_correction_end_to_end_against_oracle(torch_dev):
    # GPU raw sums + GPU solve against oracle raw sums + oracle solve. The raw sums agree
    # to the FP32 tolerance; the solve can amplify that by the condition number of M,
    # so the bound here is 100 times the FP32 bar.
    pos, w, rpos, rw = _ball_catalogs(72)
    lmax, edges = 3, np.linspace(5.0, 30.0, 6)
    nr = len(edges) - 1
    nctx, rctx, _, _ = _edge_contexts(torch_dev, pos, w, rpos, rw, lmax, edges)
    got = oracle.split_orders(nctx.edge_correct(rctx), (3, 4), lmax, nr)
    nraw, _ = oracle.npcf(pos, w, (3, 4), lmax, edges, 0.0)
    rraw, _ = oracle.npcf(rpos, rw, (3, 4), lmax, edges, 0.0)
    n = oracle.split_orders(nraw, (3, 4), lmax, nr)
    r = oracle.split_orders(rraw, (3, 4), lmax, nr)
    for N in (3, 4):
        want = oracle.edge_correct(N, lmax, nr, n[N], r[N])
        scale = np.sqrt(np.mean(want ** 2))
        err = np.max(np.abs(got[N] - want)) / scale
        assert err <= 100 * TOL_FP32, (N, err)


def _oracle_truncate(per_order, N, lmax, lmax_out):
    lam = oracle.multiplets(N, lmax)
    keep = np.all(lam <= lmax_out, axis=1)
    return per_order[keep]


def test_truncate_matches_a_context_at_the_smaller_lmax(torch_dev):
    from paper_2105_08722_gb300._lib import NPCFError
    pos, w = _catalog(1200, 90.0, 73)
    edges = np.linspace(4.0, 28.0, 6)
    for orders, allparity, lmax in (((3, 4), False, 4), ((3, 4, 5), True, 3)):
        big, zbig, _ = gpu_run(torch_dev, pos, w, orders, lmax, edges, 90.0, allparity=allparity)
        _, zsmall, _ = gpu_run(torch_dev, pos, w, orders, lmax - 1, edges, 90.0, allparity=allparity)
        cut = big.truncate(zbig, lmax - 1)
        assert cut.shape == zsmall.shape
        scale = np.sqrt(np.mean(zsmall ** 2))
        assert np.max(np.abs(cut - zsmall)) <= 1e-6 * scale
        assert np.array_equal(big.truncate(zbig, lmax), zbig)
        with pytest.raises(NPCFError):
            big.truncate(zbig, lmax + 1)
        with pytest.raises(NPCFError):
            big.truncate(zbig[:-1], lmax - 1)


def test_edge_correction_at_lmax_plus_one_truncated(torch_dev):
    # Sec. 3.3: N and R measured one lmax higher than the output, corrected, then cut
    pos, w, rpos, rw = _ball_catalogs(74)
    lmax, edges = 3, np.linspace(5.0, 30.0, 6)
    nr = len(edges) - 1
    nctx, rctx, _, _ = _edge_contexts(torch_dev, pos, w, rpos, rw, lmax + 1, edges)
    got = oracle.split_orders(nctx.truncate(nctx.edge_correct(rctx), lmax), (3, 4), lmax, nr)
    nraw, _ = oracle.npcf(pos, w, (3, 4), lmax + 1, edges, 0.0)
    rraw, _ = oracle.npcf(rpos, rw, (3, 4), lmax + 1, edges, 0.0)
    n = oracle.split_orders(nraw, (3, 4), lmax + 1, nr)
    r = oracle.split_orders(rraw, (3, 4), lmax + 1, nr)
    for N in (3, 4):
        want = _oracle_truncate(oracle.edge_correct(N, lmax + 1, nr, n[N], r[N]), N, lmax + 1, lmax)
        scale = np.sqrt(np.mean(want ** 2))
        assert np.max(np.abs(got[N] - want)) / scale <= 100 * TOL_FP32, N


def test_edge_correction_of_coadded_random_splits(torch_dev):
    # two random splits: N = (D - R1) + (D - R2) and R = R1 + R2 co-added by repeated
    # accumulate calls, then corrected (the paper's split randoms)
    torch, dev = torch_dev
    from paper_2105_08722_gb300._lib import NPCF
    pos, w, rpos, rw = _ball_catalogs(75, n_rand=3000)
    nd = int(np.sum(w > 0))
    d = pos[:nd]
    halves = (rpos[:1500], rpos[1500:])
    lmax, edges = 3, np.linspace(5.0, 30.0, 6)
    nr = len(edges) - 1
    nctx, rctx = NPCF(lmax, (3, 4), edges, 0.0), NPCF(lmax, (3, 4), edges, 0.0)
    nsum = rsum = 0.0
    for rk in halves:
        ratio = nd / len(rk)
        dm = np.concatenate([d, rk]).astype(np.float32)
        wm = np.concatenate([np.ones(nd), np.full(len(rk), -ratio)]).astype(np.float32)
        wr = np.full(len(rk), ratio, np.float32)
        nctx.accumulate(torch.from_numpy(dm).to(dev), torch.from_numpy(wm).to(dev))
        rctx.accumulate(torch.from_numpy(rk).to(dev), torch.from_numpy(wr).to(dev))
        nsum = nsum + oracle.npcf(dm, wm, (3, 4), lmax, edges, 0.0)[0]
        rsum = rsum + oracle.npcf(rk, wr, (3, 4), lmax, edges, 0.0)[0]
    got = oracle.split_orders(nctx.edge_correct(rctx), (3, 4), lmax, nr)
    n = oracle.split_orders(nsum, (3, 4), lmax, nr)
    r = oracle.split_orders(rsum, (3, 4), lmax, nr)
    for N in (3, 4):
        want = oracle.edge_correct(N, lmax, nr, n[N], r[N])
        scale = np.sqrt(np.mean(want ** 2))
        assert np.max(np.abs(got[N] - want)) / scale <= 100 * TOL_FP32, N


def test_edge_correction_rejects_mismatched_or_unsupported_contexts(torch_dev):
    from paper_2105_08722_gb300._lib import NPCF, NPCFError
    edges = np.linspace(5.0, 30.0, 6)
    a = NPCF(3, (3, 4), edges, 0.0)
    b = NPCF(2, (3, 4), edges, 0.0)
    with pytest.raises(NPCFError):
        a.edge_correct(b)
    c = NPCF(3, (3, 4), edges, 0.0, 0, True)
    with pytest.raises(NPCFError):
        c.edge_correct(c)
    d = NPCF(2, (5,), edges, 0.0)
    with pytest.raises(NPCFError):
        d.edge_correct(d)
    for x in (a, b, c, d):
        x.close()


# ------------------------------------------------------------------ survey geometry (D - R)

@pytest.fixture(scope="module")
def survey():
    return catalogs.survey_dmr_and_randoms()


def test_survey_subset_dmr_multiplets_and_edge_correction(torch_dev, survey):
    # the seeded 20k subset (4k data, 16k randoms) of the 400k + 1.6M survey catalogs:
    # raw D - R and R multiplets, then the edge-corrected ones, against the oracle
    dr, rr = catalogs.survey_subset(*survey)
    nr = len(dr.edges) - 1
    nctx, nraw, ncnt = gpu_run(torch_dev, dr.pos, dr.w, dr.orders, dr.lmax, dr.edges, 0.0)
    rctx, rraw, _ = gpu_run(torch_dev, rr.pos, rr.w, rr.orders, rr.lmax, rr.edges, 0.0)
    onraw, ocnt = oracle.npcf(dr.pos, dr.w, dr.orders, dr.lmax, dr.edges, 0.0)
    orraw, _ = oracle.npcf(rr.pos, rr.w, rr.orders, rr.lmax, rr.edges, 0.0)
    assert np.array_equal(ncnt, ocnt)
    assert_orders_close(nraw, onraw, dr.orders, dr.lmax, nr)
    assert_orders_close(rraw, orraw, rr.orders, rr.lmax, nr)
    got = oracle.split_orders(nctx.edge_correct(rctx), dr.orders, dr.lmax, nr)
    n = oracle.split_orders(onraw, dr.orders, dr.lmax, nr)
    r = oracle.split_orders(orraw, dr.orders, dr.lmax, nr)
    for N in dr.orders:
        want = oracle.edge_correct(N, dr.lmax, nr, n[N], r[N])
        err = np.max(np.abs(got[N] - want)) / np.sqrt(np.mean(want ** 2))
        assert err <= 100 * TOL_FP32, (N, err)


@pytest.mark.parametrize("prec", [0, 1])
def test_survey_full_dmr_sampled_primaries(torch_dev, survey, prec):
    # the full 2M-point D - R catalog; 24 seeded primaries (data and randoms) summed
    # against every secondary, FP32 and split-bf16 contractions
    dr, _ = survey
    rng = np.random.default_rng(3004)
    sample = np.sort(np.concatenate([rng.choice(400_000, 8, replace=False),
                                     400_000 + rng.choice(1_600_000, 16, replace=False)]))
    wp = np.zeros(dr.n, np.float32)
    wp[sample] = dr.w[sample]
    _, got, _ = gpu_run(torch_dev, dr.pos, dr.w, dr.orders, dr.lmax, dr.edges, 0.0, wprim=wp, prec=prec)
    want, _ = oracle.npcf(dr.pos, dr.w, dr.orders, dr.lmax, dr.edges, 0.0, prim=sample)
    assert_orders_close(got, want, dr.orders, dr.lmax, len(dr.edges) - 1,
                        tol=TOL_FP32 if prec == 0 else TOL_BF16)


# ------------------------------------------------------------------ batches of catalogs (a8)

def _batch_run(torch_dev, cats, ws, orders, lmax, edges, box, prec=0, repeat=1, tuning=None):
    torch, dev = torch_dev
    from paper_2105_08722_gb300._lib import NPCF
    est = NPCF(lmax, orders, edges, box, prec)
    for k, v in (tuning or {}).items():
        est.set_tuning(k, v)
    pos = torch.from_numpy(np.ascontiguousarray(np.concatenate(cats), np.float32)).to(dev)
    w = torch.from_numpy(np.ascontiguousarray(np.concatenate(ws), np.float32)).to(dev)
    off = np.concatenate([[0], np.cumsum([len(c) for c in cats])])
    stream = torch.cuda.Stream(dev)   # a capturable stream: the batch runs as a CUDA graph
    with torch.cuda.stream(stream):
        for _ in range(repeat):
            est.accumulate_batch(pos, w, off, stream=stream)
    stream.synchronize()
    return est, est.finalize_batch(), est.pair_counts_batch()


def test_batch_matches_single_catalog_runs(torch_dev):
    # catalogs of uneven size (one empty, one with a single point) in one batch: every
    # catalog's multiplets and counts equal those of its own single-catalog run
    rng = np.random.default_rng(81)
    sizes = [700, 0, 1, 2600, 1500]
    cats = [rng.uniform(0, 120.0, size=(n, 3)).astype(np.float32) for n in sizes]
    ws = [rng.uniform(0.5, 1.5, size=n).astype(np.float32) for n in sizes]
    edges = np.linspace(4.0, 30.0, 7)
    est, got, counts = _batch_run(torch_dev, cats, ws, (3, 4), 4, edges, 120.0)
    assert est.batch_info() == (len(sizes), 1)
    for k, (c, w) in enumerate(zip(cats, ws)):
        if len(c) == 0:
            assert np.all(got[k] == 0) and np.all(counts[k] == 0)
            continue
        _, want, wcounts = gpu_run(torch_dev, c, w, (3, 4), 4, edges, 120.0)
        assert np.array_equal(counts[k], wcounts), k
        scale = max(np.sqrt(np.mean(want ** 2)), 1e-300)
        assert np.max(np.abs(got[k] - want)) <= TOL_FP32 * scale, k


@pytest.mark.parametrize("orders,lmax,tuning", [
    ((5,), 3, {}),            # 5PCF with the P34 cache: chunk rows of several catalogs
    ((5,), 3, {9: 1}),        # the register-only 5PCF kernel
    ((5,), 3, {9: 2}),        # the P34 cache with the coupling terms read through L1
    ((3, 4), 4, {4: 1}),      # the high-lmax 4PCF kernel forced
])
def test_batch_of_each_contraction_kernel_matches_single_runs(torch_dev, orders, lmax, tuning):
    # every contraction kernel sums a batch's catalogs into their own chunk rows: each
    # catalog's multiplets equal those of its own run with the same kernel
    rng = np.random.default_rng(83)
    sizes = [500, 1, 1200, 0, 800]
    cats = [rng.uniform(0, 110.0, size=(n, 3)).astype(np.float32) for n in sizes]
    ws = [rng.uniform(0.5, 1.5, size=n).astype(np.float32) for n in sizes]
    edges = np.linspace(4.0, 32.0, 7)
    _, got, counts = _batch_run(torch_dev, cats, ws, orders, lmax, edges, 110.0, tuning=tuning)
    for k, (c, w) in enumerate(zip(cats, ws)):
        if len(c) == 0:
            assert np.all(got[k] == 0) and np.all(counts[k] == 0)
            continue
        _, want, wcounts = gpu_run(torch_dev, c, w, orders, lmax, edges, 110.0, tuning=tuning)
        assert np.array_equal(counts[k], wcounts), k
        scale = max(np.sqrt(np.mean(want ** 2)), 1e-300)
        assert np.max(np.abs(got[k] - want)) <= TOL_FP32 * scale, k
    # and against the oracle for the largest catalog
    want, _ = oracle.npcf(cats[2], ws[2], orders, lmax, edges, 110.0)
    assert_orders_close(got[2], want, orders, lmax, 6)


def test_batch_graph_replay_coadds_and_mode_errors(torch_dev):
    from paper_2105_08722_gb300._lib import NPCFError
    rng = np.random.default_rng(82)
    cats = [rng.uniform(0, 100.0, size=(n, 3)).astype(np.float32) for n in (900, 1300)]
    ws = [np.ones(len(c), np.float32) for c in cats]
    edges = np.linspace(4.0, 25.0, 6)
    est1, once, c1 = _batch_run(torch_dev, cats, ws, (3, 4), 3, edges, 100.0)
    est3, thrice, c3 = _batch_run(torch_dev, cats, ws, (3, 4), 3, edges, 100.0, repeat=3)
    assert est3.batch_info() == (2, 3)   # captured once, launched as a graph three times
    assert np.array_equal(c3, 3 * c1)
    assert np.max(np.abs(thrice - 3 * once)) <= 1e-12 * np.max(np.abs(once))
    with pytest.raises(NPCFError):   # a batch context is read with the batch calls
        est3.finalize()
    torch, dev = torch_dev
    single = torch.from_numpy(cats[0]).to(dev)
    with pytest.raises(NPCFError):   # one catalog into accumulators that hold two
        est3.accumulate(single, torch.ones(len(cats[0]), device=dev))
    est3.reset()
    est3.accumulate(single, torch.ones(len(cats[0]), device=dev))
    assert est3.batch_info()[0] == 1


@pytest.mark.parametrize("prec", [0, 1])
def test_lognormal_batch_against_oracle(torch_dev, prec):
    # three log-normal periodic catalogs of different sizes in one batch, each against the
    # oracle; FP32 and split-bf16 contractions
    cats = [catalogs.lognormal_box(n, 300.0, 32, seed=5100 + n) for n in (1200, 2500, 1800)]
    ws = [np.ones(len(c), np.float32) for c in cats]
    edges = np.linspace(8.0, 60.0, 9)
    _, got, counts = _batch_run(torch_dev, cats, ws, (3, 4), 4, edges, 300.0, prec=prec)
    for k, c in enumerate(cats):
        want, wcounts = oracle.npcf(c, ws[k], (3, 4), 4, edges, 300.0)
        assert np.array_equal(counts[k], wcounts), k
        assert_orders_close(got[k], want, (3, 4), 4, 8, tol=TOL_FP32 if prec == 0 else TOL_BF16)


def test_autotune_picks_candidates_and_leaves_sums_empty(torch_dev):
    torch, dev = torch_dev
    from paper_2105_08722_gb300._lib import NPCF
    pos = catalogs.lognormal_box(20000, 500.0, 64, seed=91)
    w = np.ones(len(pos), np.float32)
    edges = np.linspace(10.0, 80.0, 8)
    tp, tw = torch.from_numpy(pos).to(dev), torch.from_numpy(w).to(dev)
    est = NPCF(4, (3, 4), edges, 500.0)
    chosen = est.autotune(tp, tw)
    assert chosen["cells_per_rmax"] in (2, 3, 4, 5, 6) and chosen["pair_chunk"] in (8, 16, 32, 64)
    assert chosen["pair_cap"] in (4096, 8192) and chosen["chunk"] >= 64
    assert est.batch_info()[0] == 0 and np.all(est.finalize() == 0)
    est.accumulate(tp, tw)
    got = est.finalize()
    _, want, _ = gpu_run(torch_dev, pos, w, (3, 4), 4, edges, 500.0)
    assert np.max(np.abs(got - want)) <= TOL_FP32 * np.sqrt(np.mean(want ** 2))


def test_batched_mocks_full_size_sampled_primaries(torch_dev):
    # the 64-catalog workload (6.46M points, split-bf16 as in the bench) in one batch; two
    # seeded primaries in each of 8 catalogs are summed against their full catalogs and
    # compared with the oracle; every other catalog has no primary and stays zero
    torch, dev = torch_dev
    from paper_2105_08722_gb300._lib import NPCF
    cats, edges = catalogs.batch64_lognormal()
    sizes = np.array([len(c) for c in cats])
    off = np.concatenate([[0], np.cumsum(sizes)])
    rng = np.random.default_rng(5005)
    picked = np.sort(rng.choice(len(cats), 8, replace=False))
    wp = np.zeros(off[-1], np.float32)
    samples = {}
    for k in picked:
        samples[k] = np.sort(rng.choice(sizes[k], 2, replace=False))
        wp[off[k] + samples[k]] = 1.0
    pos = torch.from_numpy(np.ascontiguousarray(np.concatenate(cats), np.float32)).to(dev)
    w = torch.ones(off[-1], device=dev)
    est = NPCF(5, (3, 4), edges, 1000.0, 1)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        est.accumulate_batch(pos, w, off, wprim=torch.from_numpy(wp).to(dev), stream=stream)
    stream.synchronize()
    got = est.finalize_batch()
    for k in range(len(cats)):
        if k not in samples:
            assert np.all(got[k] == 0), k
            continue
        want, _ = oracle.npcf(cats[k], np.ones(sizes[k], np.float32), (3, 4), 5, edges, 1000.0, prim=samples[k])
        assert_orders_close(got[k], want, (3, 4), 5, 10, tol=TOL_BF16)
