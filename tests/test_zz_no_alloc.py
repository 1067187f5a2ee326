"""osp_topk_noalloc (scratch in a fixed device array, no allocation) against
osp_topk on the same scores, on consecutive calls. Collected last on purpose:
it must pass alone and after every other test has used the device."""
import numpy as np
import pytest

from paper_1712_00595_gb300 import native as N
from paper_1712_00595_gb300 import workloads as W

C_RESTART = 0.15


def _graph_with_ties(n=3000, seed=8):
    # a star with 700 equal-score leaves (ties), a random part, unreachable nodes
    rng = np.random.default_rng(seed)
    src = [0] * 700 + list(rng.integers(701, n, 8000)) + [5, 9]
    dst = list(range(1, 701)) + list(rng.integers(701, n, 8000)) + [801, 802]
    src, dst = np.array(src, np.int32), np.array(dst, np.int32)
    keep = src != dst
    return n, src[keep], dst[keep]


def _rmat_graph(scale=17, m=1 << 20):
    _, src, dst = W.rmat_graph(scale, m, seed=W.BASE_SEED + 31)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    return 1 << scale, src.astype(np.int32), dst.astype(np.int32)


class _Out:
    """Device output buffers for up to k_max entries, made once by the test."""

    def __init__(self, torch, k_max=4096):
        self.torch = torch
        self.ids = torch.empty(k_max, dtype=torch.int32, device="cuda:0")
        self.sc = torch.empty(k_max, dtype=torch.float64, device="cuda:0")
        self.got = torch.empty(1, dtype=torch.int32, device="cuda:0")

    def run(self, r_dev, k, normalize):
        self.ids.fill_(-1)
        self.sc.fill_(-1.0)
        self.got.fill_(-1)
        self.torch.cuda.synchronize()
        N.topk_noalloc(r_dev, r_dev.numel(), k, self.ids, self.sc, self.got, normalize=normalize)
        self.torch.cuda.synchronize()

    def result(self):
        kk = int(self.got.item())
        return self.ids[:kk].cpu().numpy(), self.sc[:kk].cpu().numpy()


def _noalloc(torch, r_dev, k, normalize):
    out = _Out(torch)
    out.run(r_dev, k, normalize)
    return out.result()


def test_rejects_sizes_beyond_the_maximum():
    # every argument check runs before any CUDA call, so this needs no device
    N.load_library()
    fake = 256
    for n, k in ((N.TOPK_NOALLOC_MAX_N + 1, 10), (-1, 10), (100, 0), (100, 4097)):
        with pytest.raises(N.OspError) as e:
            N.topk_noalloc(fake, n, k, fake, fake, fake)
        assert e.value.status == N.OSP_EINVAL
        assert str(N.TOPK_NOALLOC_MAX_N) in str(e.value)


@pytest.mark.gpu
@pytest.mark.parametrize("make", [_graph_with_ties, _rmat_graph])
def test_noalloc_matches_osp_topk_on_consecutive_calls(make):
    torch = pytest.importorskip("torch")
    n, src, dst = make()
    eng = N.Engine(precision=N.OSP_PREC_FP64, device=0)
    eng.load_graph(n, src, dst)
    eng.set_seeds([0], C_RESTART)
    eng.init_scores(1e-12)
    torch.cuda.set_device(0)
    r_dev = torch.empty(n, dtype=torch.float64, device="cuda:0")
    eng.query_device(r_dev, normalize=False)
    torch.cuda.synchronize()
    out = _Out(torch)
    # the set-up call: it looks the array up and, under CUDA's lazy module
    # loading, loads the module holding it (device memory taken once)
    out.run(r_dev, 16, False)
    # two calls in a row per case
    for k, normalize in ((4096, False), (701, False), (100, True), (1, True), (4096, True)):
        want_ids, want_sc = eng.topk(k, normalize=normalize)
        for call in range(2):
            free0 = torch.cuda.mem_get_info(0)[0]
            allocs0 = torch.cuda.memory_stats(0).get("allocation.all.allocated", 0)
            out.run(r_dev, k, normalize)
            free1 = torch.cuda.mem_get_info(0)[0]
            allocs1 = torch.cuda.memory_stats(0).get("allocation.all.allocated", 0)
            ids, sc = out.result()
            assert np.array_equal(ids, want_ids), (k, normalize, call)
            if normalize:
                # both sides divide by an atomically summed norm: equal up to its rounding
                assert np.allclose(sc, want_sc, rtol=1e-14, atol=0)
            else:
                assert np.array_equal(sc, want_sc)
            # nothing on the device was allocated by the call itself: no new
            # allocation in this process (torch's allocator counts), and the
            # device's free memory unchanged (this assumes no other context is
            # allocating on the GPU meanwhile)
            assert allocs1 == allocs0, (k, normalize, call)
            assert free1 == free0, (k, normalize, call)
    eng.close()


@pytest.mark.gpu
def test_noalloc_short_vectors():
    torch = pytest.importorskip("torch")
    torch.cuda.set_device(0)
    r = torch.tensor([0.5, 0.25, 0.25, 0.0, 0.75, 0.25, 0.125], dtype=torch.float64,
                     device="cuda:0")
    ids, sc = _noalloc(torch, r, 20, False)
    assert ids.tolist() == [4, 0, 1, 2, 5, 6, 3]
    assert sc.tolist() == [0.75, 0.5, 0.25, 0.25, 0.25, 0.125, 0.0]
    ids, sc = _noalloc(torch, r, 3, True)
    assert ids.tolist() == [4, 0, 1]
    assert np.allclose(sc, np.array([0.75, 0.5, 0.25]) / 2.125, rtol=1e-15, atol=0)
    empty = torch.empty(0, dtype=torch.float64, device="cuda:0")
    ids, sc = _noalloc(torch, empty, 5, False)
    assert ids.size == 0 and sc.size == 0


@pytest.mark.gpu
@pytest.mark.parametrize("n", [N.TOPK_NOALLOC_MAX_N, N.TOPK_NOALLOC_MAX_N - 1])
def test_noalloc_at_the_size_limit(n):
    """The largest vectors accepted (the last chunk full or partial): a seeded
    random vector with planted ties, against a host sort by (score desc, id
    asc), twice in a row."""
    torch = pytest.importorskip("torch")
    torch.cuda.set_device(0)
    rng = np.random.default_rng(n)
    r = rng.random(n)
    r[rng.choice(n, 5000, replace=False)] = 0.999999  # ties inside the top k
    r[n - 3:] = 1.5  # the last ids rank first
    order = np.lexsort((np.arange(n), -r))
    r_dev = torch.from_numpy(r).to("cuda:0")
    out = _Out(torch)
    for k in (4096, 100):
        for _ in range(2):
            out.run(r_dev, k, False)
            ids, sc = out.result()
            assert np.array_equal(ids, order[:k].astype(np.int32))
            assert np.array_equal(sc, r[order[:k]])
