"""GPU parity of the batched persistent launch: every instance of a mixed
dense + tet batch equals its single-instance oracle result; graph replays after
the inputs change and after the buffer pointers change."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2507_13204_gb300 import workloads as W
from tests.helpers import TOL, f32_round, rel_l2, rel_scalar

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api(cuda_ok):
    from paper_2507_13204_gb300 import build
    build.build()
    from paper_2507_13204_gb300 import api as A
    return A


def _make(api, dtype, dense_ns, tet_boxes, seed=0):
    td = torch.float64 if dtype == "f64" else torch.float32
    rnd = (lambda a: a) if dtype == "f64" else f32_round
    probs, host, xs, fs, gxs = [], [], [], [], []
    for k, n in enumerate(dense_ns):
        A, x = W.quadform_inputs(n, seed=seed + k)
        A, x = rnd(A), rnd(x)
        p = api.QuadForm(torch.tensor(A, dtype=td, device="cuda"))
        probs.append(p)
        host.append(("dense", A, x))
        xs.append(torch.tensor(x, dtype=td, device="cuda"))
    for k, box in enumerate(tet_boxes):
        mesh, u = W.batched_tet_instance(k, box)
        G, u = rnd(mesh.G), rnd(u)
        p = api.TetEnergy(torch.tensor(mesh.conn, device="cuda"),
                          torch.tensor(G, dtype=td, device="cuda"), mesh.nv)
        probs.append(p)
        host.append(("tet", mesh.conn, G, u))
        xs.append(torch.tensor(u, dtype=td, device="cuda"))
    for x in xs:
        fs.append(torch.empty((), dtype=td, device="cuda"))
        gxs.append(torch.full_like(x, 3.0))
    return probs, host, xs, fs, gxs


def _oracle(h):
    if h[0] == "dense":
        return O.quadform_grad(h[1], h[2])
    return O.tet_grad(h[1], h[2], h[3])


DENSE = [32, 33, 64, 100, 255, 256, 257, 511, 1000, 1024, 1500, 2047, 2048]
BOXES = [(1, 1, 1), (3, 3, 2), (5, 5, 7), (10, 10, 12)]


@pytest.mark.parametrize("strategy", ["auto", "warp"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_matches_oracle_per_instance(api, dtype, strategy, tmp_path, monkeypatch):
    monkeypatch.setenv("KG_TUNE_CACHE", str(tmp_path / "tune.json"))
    probs, host, xs, fs, gxs = _make(api, dtype, DENSE, BOXES)
    batch = api.Batch(probs, strategy=strategy)
    batch.grad(xs, fs, gxs)
    batch.sync()
    tol = TOL[dtype]
    for h, f, g in zip(host, fs, gxs):
        f_ref, g_ref = _oracle(h)
        assert rel_scalar(f.item(), f_ref) <= tol, h[0]
        assert rel_l2(g.cpu().numpy(), g_ref) <= tol, h[0]
    assert (tmp_path / "tune.json").exists()
    # the per-instance launch loop gives the same results
    fl = [torch.empty_like(f) for f in fs]
    gl = [torch.empty_like(g) for g in gxs]
    batch.grad_loop(xs, fl, gl)
    torch.cuda.synchronize()
    for g, h2 in zip(gxs, gl):
        assert rel_l2(h2.cpu().numpy(), g.cpu().numpy()) <= tol


def test_graph_replay_after_inputs_and_pointers_change(api, tmp_path, monkeypatch):
    monkeypatch.setenv("KG_TUNE_CACHE", str(tmp_path / "tune.json"))
    probs, host, xs, fs, gxs = _make(api, "f64", [64, 700, 2000], [(4, 4, 4)], seed=5)
    batch = api.Batch(probs)
    batch.grad(xs, fs, gxs)
    first = [g.clone() for g in gxs]
    batch.grad(xs, fs, gxs)  # replay: dense results are bitwise reproducible
    torch.cuda.synchronize()
    for a, b, h in zip(first, gxs, host):
        if h[0] == "dense":
            assert torch.equal(a, b)
    # mutate x in place and replay
    for x in xs:
        x.mul_(0.5)
    batch.grad(xs, fs, gxs)
    batch.sync()
    for h, x, f, g in zip(host, xs, fs, gxs):
        hx = x.cpu().numpy()
        ref = O.quadform_grad(h[1], hx) if h[0] == "dense" else O.tet_grad(h[1], h[2], hx)
        assert rel_scalar(f.item(), ref[0]) <= TOL["f64"]
        assert rel_l2(g.cpu().numpy(), ref[1]) <= TOL["f64"]
    # new buffers (pointer tables change): the descriptors are refreshed
    xs2 = [x.clone() * 2 for x in xs]
    gxs2 = [torch.empty_like(g) for g in gxs]
    batch.grad(xs2, fs, gxs2)
    batch.sync()
    for h, x, g in zip(host, xs2, gxs2):
        hx = x.cpu().numpy()
        ref = O.quadform_grad(h[1], hx) if h[0] == "dense" else O.tet_grad(h[1], h[2], hx)
        assert rel_l2(g.cpu().numpy(), ref[1]) <= TOL["f64"]
    # bound buffers (pointer tables built once): the same results, then again after an
    # in-place change of x; mixing the two call forms is an error
    bound = batch.bind(xs2, fs, gxs2)
    before = [g.clone() for g in gxs2]
    batch.grad(bound)
    batch.sync()
    for a, b, h in zip(before, gxs2, host):
        if h[0] == "dense":
            assert torch.equal(a, b)
    for x in xs2:
        x.mul_(-1.0)
    batch.grad(bound)
    batch.sync()
    for h, x, g in zip(host, xs2, gxs2):
        hx = x.cpu().numpy()
        ref = O.quadform_grad(h[1], hx) if h[0] == "dense" else O.tet_grad(h[1], h[2], hx)
        assert rel_l2(g.cpu().numpy(), ref[1]) <= TOL["f64"]
    with pytest.raises(ValueError):
        batch.grad(bound, fs, gxs2)


def test_batch_rejects_bad_inputs(api):
    from paper_2507_13204_gb300 import _lib as L
    big = api.QuadForm(torch.zeros((4, 4096), dtype=torch.float64, device="cuda"))
    with pytest.raises(L.KGError) as ei:
        api.Batch([big])
    assert ei.value.status == L.KG_ERR_UNSUPPORTED
    a = api.QuadForm(torch.zeros((8, 8), dtype=torch.float64, device="cuda"))
    b = api.QuadForm(torch.zeros((8, 8), dtype=torch.float32, device="cuda"))
    with pytest.raises(L.KGError) as ei:
        api.Batch([a, b])
    assert ei.value.status == L.KG_ERR_INVALID_ARG


def _bucket(v):
    return int(v).bit_length() - 1  # floor(log2 v), the library's size bucket


def _items(dense_ns, tet_nes, rows, elems):
    """Work items of a batch whose tiles are rows[bucket] rows (dense) and
    elems[bucket] elements (tet), one item per tile."""
    return (sum(-(-n // rows[_bucket(n)]) for n in dense_ns)
            + sum(-(-ne // elems[_bucket(ne)]) for ne in tet_nes))


def test_full_4096_dense_512_tet_batch_sampled_against_oracle(api, tmp_path, monkeypatch):
    """The benchmarked batch (4096 dense instances, n log-uniform in [32, 2048],
    A drawn on the device, plus 512 tet meshes of 1e3..1e5 elements), one
    kg_grad_batched launch; sampled instances against the oracle: one dense
    instance per size bucket (first and last of each), the smallest and the
    largest n, the 8 largest and the smallest tet meshes, and the last instance.
    Then the tuning cache: a second batch reads the tiles back per bucket."""
    import json
    monkeypatch.setenv("KG_TUNE_CACHE", str(tmp_path / "tune.json"))
    dev = torch.device("cuda", 0)
    sizes = [int(n) for n in W.batched_dense_sizes(4096)]
    boxes = W.batched_tet_boxes(512)
    probs, dense_dev, tets, nx = [], [], [], []
    for k, n in enumerate(sizes):
        A, x = W.batched_dense_device(k, n, dev)
        dense_dev.append((A, x))
        probs.append(api.QuadForm(A))
        nx.append(n)
    for k, box in enumerate(boxes):
        mesh, u = W.batched_tet_instance(k, box)
        conn, G = torch.tensor(mesh.conn, device=dev), torch.tensor(mesh.G, device=dev)
        tets.append((mesh, u, conn, G))
        probs.append(api.TetEnergy(conn, G, mesh.nv))
        nx.append(mesh.nv)
    xs = [x for _, x in dense_dev] + [torch.tensor(t[1], device=dev) for t in tets]
    fs = [torch.empty((), dtype=torch.float64, device=dev) for _ in nx]
    gxs = [torch.full((v,), 5.0, dtype=torch.float64, device=dev) for v in nx]
    batch = api.Batch(probs)
    arith, nitems, _ = batch.config
    batch.grad(xs, fs, gxs)
    batch.sync()

    # the sample
    by_bucket = {}
    for k, n in enumerate(sizes):
        by_bucket.setdefault(_bucket(n), []).append(k)
    assert sorted(by_bucket) == list(range(5, 12))
    dense_ids = {ks[0] for ks in by_bucket.values()} | {ks[-1] for ks in by_bucket.values()}
    dense_ids |= {int(np.argmin(sizes)), int(np.argmax(sizes))}
    nes = [t[0].ne for t in tets]
    order = np.argsort(nes, kind="stable")
    tet_ids = {int(j) for j in order[-8:]} | {int(order[0]), len(tets) - 1}
    assert max(nes) > 90_000
    for k in sorted(dense_ids):
        A, x = dense_dev[k]
        f_ref, g_ref = O.quadform_grad(A.cpu().numpy(), x.cpu().numpy())
        assert rel_scalar(fs[k].item(), f_ref) <= TOL["f64"], (k, sizes[k])
        assert rel_l2(gxs[k].cpu().numpy(), g_ref) <= TOL["f64"], (k, sizes[k])
    for j in sorted(tet_ids):
        mesh, u, _, _ = tets[j]
        f_ref, g_ref = O.tet_grad(mesh.conn, mesh.G, u)
        i = len(sizes) + j
        assert rel_scalar(fs[i].item(), f_ref) <= TOL["f64"], (j, mesh.ne)
        assert rel_l2(gxs[i].cpu().numpy(), g_ref) <= TOL["f64"], (j, mesh.ne)

    # the tuning cache holds one entry per (kind, bucket), and the work table follows it
    cache = json.loads((tmp_path / "tune.json").read_text())
    key = lambda kind, b: next(k for k in cache if k.endswith(f"|{arith}|{kind}|{b}"))
    dense_b = sorted({_bucket(n) for n in sizes})
    tet_b = sorted({_bucket(ne) for ne in nes})
    rows = {b: cache[key("dense", b)] for b in dense_b}
    elems = {b: cache[key("tet", b)] for b in tet_b}
    assert nitems == _items(sizes, nes, rows, elems)
    # a second batch over the same problems reads the tiles back from the cache
    for r, e in ((4, 1024), (128, 16384)):
        for b in dense_b:
            cache[key("dense", b)] = r
        for b in tet_b:
            cache[key("tet", b)] = e
        (tmp_path / "tune.json").write_text(json.dumps(cache, indent=2))  # one entry a line
        second = api.Batch(probs)
        assert second.config[1] == _items(sizes, nes, {b: r for b in dense_b},
                                          {b: e for b in tet_b})
        second.close()
    batch.close()
    for p in probs:
        p.close()


def test_batch_float_pair_copies_budget(api, tmp_path, monkeypatch):
    # dense instances without their own float-pair copy (n < 1024) get one from the batch,
    # largest first, within the budget; the copy holds the same pairs as the per-load
    # split, so with the same tiles the results agree bitwise.  Odd n: an odd element count.
    monkeypatch.setenv("KG_NO_AUTOTUNE", "1")
    ns = [33, 255, 257, 511, 1000, 1024]
    probs, host, xs, fs, gxs = _make(api, "f64", ns, [(3, 3, 2)], seed=11)
    outs = []
    for budget in (0, 1, 8 * 1000 * 1000 + 8):  # all, none, only the n = 1000 instance
        batch = api.Batch(probs, budget_bytes=budget)
        assert batch.config[0] == "pair"
        f2 = [torch.empty_like(f) for f in fs]
        g2 = [torch.full_like(g, 3.0) for g in gxs]
        batch.grad(xs, f2, g2)
        batch.sync()
        for h, f, g in zip(host, f2, g2):
            f_ref, g_ref = _oracle(h)
            assert rel_scalar(f.item(), f_ref) <= TOL["f64"], h[0]
            assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f64"], h[0]
        outs.append([g.cpu().numpy() for g in g2[:len(ns)]])
        batch.close()
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert np.array_equal(a, b)


def test_batch_range_scan_sees_the_last_of_an_odd_count(api, tmp_path, monkeypatch):
    # 33 x 33 = 1089 entries: the last one, below the pair range, makes the batch native
    monkeypatch.setenv("KG_NO_AUTOTUNE", "1")
    A, x = W.quadform_inputs(33, seed=2)
    A[-1, -1] = 2.0 ** -70
    p = api.QuadForm(torch.tensor(A, device="cuda"))
    batch = api.Batch([p])
    assert batch.config[0] == "native"
    f = torch.empty((), dtype=torch.float64, device="cuda")
    g = torch.empty(33, dtype=torch.float64, device="cuda")
    batch.grad([torch.tensor(x, device="cuda")], [f], [g])
    batch.sync()
    f_ref, g_ref = O.quadform_grad(A, x)
    assert rel_scalar(f.item(), f_ref) <= TOL["f64"]
    assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f64"]
    batch.close()
    p.close()


def test_batch_tiny_and_odd_rows_through_the_ring(api, tmp_path, monkeypatch):
    # rows of 8 .. 136 bytes: chunk starts 8 bytes off the 16-byte boundary (odd n), several
    # chunks in one tile, instances of one row; in pair arithmetic on the batch's copies
    monkeypatch.setenv("KG_TUNE_CACHE", str(tmp_path / "tune.json"))
    ns = [1, 2, 3, 5, 7, 9, 17, 31]
    probs, host, xs, fs, gxs = _make(api, "f64", ns, [], seed=21)
    batch = api.Batch(probs)
    assert batch.config[0] == "pair"
    batch.grad(xs, fs, gxs)
    batch.sync()
    for h, f, g in zip(host, fs, gxs):
        f_ref, g_ref = _oracle(h)
        assert rel_scalar(f.item(), f_ref) <= TOL["f64"]
        assert rel_l2(g.cpu().numpy(), g_ref) <= TOL["f64"]
    batch.close()
