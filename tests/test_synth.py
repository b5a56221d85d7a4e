"""The synthetic inputs follow their stated recipe (stand-ins for the
paper's daily bitcoin graphs, Section 2 and Section 4): inputs per
transaction Geometric(1/2) on 1..20, outputs 2 with probability 0.7 else
Geometric(1/2) on 1..50, each endpoint reusing an existing address with
probability 0.4 (Zipf over creation rank, so the oldest address is the most
reused), else a new one; forests of random recursive trees with about 10 %
extra edges and log-uniform sizes.  Checked statistically on the 200k-
transaction workload and the batched-component forest."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

import synth


@pytest.fixture(scope="module")
def c2():
    return synth.tx_lists(**synth.C2)


def test_transaction_list_shapes(c2):
    assert c2.n_tx == 200_000
    assert c2.in_off[0] == 0 and c2.out_off[0] == 0
    assert c2.in_off[-1] == len(c2.in_addr) and c2.out_off[-1] == len(c2.out_addr)
    assert np.all(np.diff(c2.in_off) >= 1) and np.all(np.diff(c2.out_off) >= 1)


def test_input_counts_are_truncated_geometric(c2):
    k = np.diff(c2.in_off)
    assert k.max() <= 20
    # P(k) = 2^-k / (1 - 2^-20) for k = 1..20
    for v in (1, 2, 3):
        assert abs(np.mean(k == v) - 2.0 ** -v) < 0.01, v
    assert abs(k.mean() - 2.0) < 0.02


def test_output_counts_mix_two_and_geometric(c2):
    k = np.diff(c2.out_off)
    assert k.max() <= 50
    assert abs(np.mean(k == 2) - (0.7 + 0.3 * 0.25)) < 0.01
    assert abs(np.mean(k == 1) - 0.3 * 0.5) < 0.01
    assert abs(np.mean(k == 3) - 0.3 * 0.125) < 0.01


def test_address_reuse_rate_and_preference(c2):
    ends = len(c2.in_addr) + len(c2.out_addr)
    assert abs(1.0 - c2.n_addr_created / ends - 0.4) < 0.005
    keys = np.concatenate([c2.in_addr, c2.out_addr])
    uniq, counts = np.unique(keys, return_counts=True)
    assert len(uniq) == c2.n_addr_created
    # the first endpoint ever drawn is the oldest address (rank 1), which
    # Zipf(1.2) favours at every draw: it is the most reused one
    first = c2.in_addr[0]
    assert counts[np.searchsorted(uniq, first)] == counts.max()
    # heavy tail: a few addresses take a large share of the reuse draws
    top = np.sort(counts)[::-1]
    assert top[0] > 1000 and top[0] > 10 * top[100]


def test_forest_recipe():
    sizes, u, v = synth.forest(**synth.C3_SMALL)
    assert len(sizes) == 100_000
    assert sizes.min() >= 3 and sizes.max() <= 200
    # log-uniform: the median is the geometric mean of the bounds
    assert abs(np.median(sizes) - math.sqrt(3 * 200)) < 1.5
    extra = np.minimum(np.floor(0.1 * (sizes - 1) + 0.5), sizes * (sizes - 1) // 2 - (sizes - 1))   # round half up
    assert len(u) == int(np.sum(sizes - 1 + extra))
    n = int(sizes.sum())
    assert np.all(u != v)
    g = sp.coo_matrix((np.ones(len(u)), (u, v)), shape=(n, n)).tocsr()
    nc, lab = connected_components(g, directed=False)
    assert nc == len(sizes)                                  # every component connected, none merged
    starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    assert np.array_equal(lab[starts], np.arange(len(sizes)))  # consecutive ids per component
    # no edge twice (as an unordered pair): the extra edges join nodes not already adjacent
    lo, hi = np.minimum(u, v).astype(np.int64), np.maximum(u, v).astype(np.int64)
    assert len(np.unique(lo << 32 | hi)) == len(u)
    # each component starts with its random recursive tree: node k attaches to some j < k
    e0 = np.concatenate([[0], np.cumsum(sizes - 1 + extra)[:-1]]).astype(np.int64)
    for c in range(0, len(sizes), 997):
        k = np.arange(1, sizes[c])
        assert np.array_equal(v[e0[c] + k - 1], starts[c] + k)
        assert np.all(u[e0[c] + k - 1] >= starts[c]) and np.all(u[e0[c] + k - 1] < starts[c] + k)


def test_forest_of_given_sizes_follows_the_same_recipe():
    sizes, u, v = synth.forest(17, 300, 3.0, 200.0)
    s2, u2, v2 = synth.forest_of_sizes(17, sizes)
    assert np.array_equal(s2, sizes) and np.array_equal(u2, u) and np.array_equal(v2, v)
    want = [1, 2, 3, 4, 5, 8, 9, 16, 17, 32, 33, 255]
    s3, u3, v3 = synth.forest_of_sizes(23, want)
    n = int(s3.sum())
    g = sp.coo_matrix((np.ones(len(u3)), (u3, v3)), shape=(n, n)).tocsr()
    nc, lab = connected_components(g, directed=False)
    assert nc == len(want) and np.array_equal(np.bincount(lab), want)


def test_generator_splitmix64_matches_published_vectors():
    """The generator's SplitMix64 against the same published vectors as the
    oracle's (tests/golden/splitmix64.json)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "splitmix64.json")))
    for v in g["vectors"]:
        got = synth.splitmix64_stream(v["seed"], 3)
        if "outputs_hex" in v:
            assert [f"{int(x):016x}" for x in got] == v["outputs_hex"]
        else:
            assert [str(int(x)) for x in got] == v["outputs_dec"]


@pytest.mark.parametrize("N", [1, 2, 12, 1000])
def test_zipf_sampler_follows_the_exact_law(N):
    """Rejection-inversion Zipf(1.2) on {1..N} against P(k) = k^-1.2 / H:
    a chi-square test over the first 30 values and the tail beyond (fixed
    seed, 400,000 draws, rejected at p < 1e-6), and the law's mean."""
    stats = pytest.importorskip("scipy.stats")
    n = 400_000
    x = synth.zipf_sample(77 + N, N, n)
    assert x.min() >= 1 and x.max() <= N
    k = np.arange(1, N + 1, dtype=np.float64)
    p = k ** -1.2
    p /= p.sum()
    if N == 1:
        assert np.all(x == 1)
        return
    m = min(N, 30)
    obs = np.bincount(x, minlength=N + 1)[1:]
    o = np.append(obs[:m], obs[m:].sum()) if N > m else obs
    e = np.append(p[:m], p[m:].sum()) * n if N > m else p * n
    chi2 = float(((o - e) ** 2 / e).sum())
    assert stats.chi2.sf(chi2, len(o) - 1) > 1e-6, chi2
    mean = float((k * p).sum())
    sd = float(np.sqrt((k * k * p).sum() - mean * mean))
    assert abs(x.mean() - mean) < 6 * sd / np.sqrt(n)
