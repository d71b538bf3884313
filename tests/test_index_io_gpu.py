"""Checkpoint and in-library training of the IVFADC index.

* gbk_ivfpq_save / gbk_ivfpq_load: a loaded index returns bit-identical searches (plain,
  batched, re-ranked) and exports the same quantizers, lists, codes and ids; vectors added
  after loading land where they would in the saved index.
* gbk_nprobe_labels / gbk_nprobe_mlp_train: the recall counts equal the overlap of each
  class's search with the exact neighbours, the labels follow the rule stated in the
  header (smallest class reaching min(ceil(target k), the query's ceiling)), and training
  lowers the loss; seeded runs are reproducible."""
import numpy as np
import pytest
import torch

from paper_1702_08734_gb300 import datagen

pytestmark = pytest.mark.gpu


def _build(gbk, keep=True, rotate=False, d=64, nlist=128, M=16, n=30000, seed=500):
    cen = datagen.mixture_centres(seed, 256, d)
    x = torch.from_numpy(datagen.mixture_points(cen, seed + 1, n)).cuda()
    ix = gbk.IVFPQIndex(d, nlist, M)
    if rotate:
        q, _ = np.linalg.qr(datagen.gaussian_matrix(seed + 2, d, d).astype(np.float64))
        ix.set_rotation(torch.from_numpy(q.astype(np.float32)).cuda())
    nt = min(20000, n)
    ix.train(x[:nt], niter=6, coarse_init=datagen.permutation_prefix(seed + 3, nt, nlist),
             pq_init=datagen.permutation_prefix(seed + 4, nt, 256))
    if keep:
        ix.keep_vectors()
    ix.add(x)
    xq = torch.from_numpy(datagen.mixture_points(cen, seed + 5, 500)).cuda()
    return ix, x, xq, cen


@pytest.mark.parametrize("keep,rotate", [(False, False), (True, True)])
def test_save_load_round_trip(gbk, tmp_path, keep, rotate):
    ix, x, xq, cen = _build(gbk, keep=keep, rotate=rotate)
    path = str(tmp_path / "index.gbk")
    ix.save(path)
    lx = gbk.IVFPQIndex.load(path)
    assert lx.ntotal == ix.ntotal and (lx.d, lx.nlist, lx.M) == (ix.d, ix.nlist, ix.M)
    a, b = ix.export(), lx.export()
    for key in ("coarse", "pq", "list_off", "codes", "ids"):
        np.testing.assert_array_equal(a[key], b[key])
    for k, nprobe in ((1, 1), (10, 8), (100, 32)):
        D0, I0 = ix.search(xq, k, nprobe)
        D1, I1 = lx.search(xq, k, nprobe)
        assert torch.equal(I0, I1) and torch.equal(D0, D1)
    kq = torch.from_numpy(np.array([1, 10, 100])[datagen.randint(506, 0, 500, 3)]).to(torch.int32).cuda()
    npq = torch.from_numpy(np.array([2, 8, 32])[datagen.randint(507, 0, 500, 3)]).to(torch.int32).cuda()
    r0 = gbk.ivfpq_search_batched(ix, xq, kq, 100, npq, 32)
    r1 = gbk.ivfpq_search_batched(lx, xq, kq, 100, npq, 32)
    assert torch.equal(r0[0], r1[0]) and torch.equal(r0[1], r1[1])
    if keep:
        D0, I0 = ix.search_refine(xq, 10, 8, 64)
        D1, I1 = lx.search_refine(xq, 10, 8, 64)
        assert torch.equal(I0, I1) and torch.equal(D0, D1)
    # adding after loading = adding to the saved index
    more = torch.from_numpy(datagen.mixture_points(cen, 508, 3000)).cuda()
    ids = torch.arange(10**6, 10**6 + 3000, device="cuda")
    ix.add(more, ids=ids)
    lx.add(more, ids=ids)
    D0, I0 = ix.search(xq, 20, 16)
    D1, I1 = lx.search(xq, 20, 16)
    assert torch.equal(I0, I1) and torch.equal(D0, D1)


def test_load_rejects_bad_files(gbk, tmp_path):
    p = tmp_path / "bad.gbk"
    p.write_bytes(b"not an index" * 20)
    with pytest.raises(gbk.GbkError):
        gbk.IVFPQIndex.load(str(p))
    ix, _, _, _ = _build(gbk, keep=False, n=5000, nlist=16)
    good = tmp_path / "good.gbk"
    ix.save(str(good))
    data = good.read_bytes()
    trunc = tmp_path / "trunc.gbk"
    trunc.write_bytes(data[:len(data) // 2])
    with pytest.raises(gbk.GbkError):
        gbk.IVFPQIndex.load(str(trunc))
    with pytest.raises(gbk.GbkError):
        gbk.IVFPQIndex.load(str(tmp_path / "missing.gbk"))


def _rule(C, target, k):
    need = int(np.ceil(target * k - 1e-9))
    goal = np.minimum(need, C[-1])
    return np.argmax(C >= goal[None, :], axis=0).astype(np.int32)


@pytest.mark.parametrize("kprime", [0, 40])
def test_nprobe_labels_follow_their_definition(gbk, kprime):
    ix, x, xq, cen = _build(gbk, keep=True)
    nq, k, C = xq.shape[0], 10, 8
    lab, cnt = gbk.nprobe_labels(ix, xq, counts=True, n_classes=C, k=k, kprime=kprime)
    _, gt = gbk.knn_brute(xq, x, k)  # exact neighbours (tested against the oracle elsewhere)
    gt = gt.cpu().numpy()
    for c in range(C):
        tau = min(1 << c, ix.nlist)
        if kprime:
            _, I = ix.search_refine(xq, k, tau, kprime)
        else:
            _, I = ix.search(xq, k, tau)
        I = I.cpu().numpy()
        ov = np.array([len(set(I[q][I[q] >= 0]) & set(gt[q])) for q in range(nq)])
        np.testing.assert_array_equal(cnt[c].cpu().numpy(), ov)
    np.testing.assert_array_equal(lab.cpu().numpy(), _rule(cnt.cpu().numpy(), 0.95, k))
    # ground truth given instead of computed from the kept vectors: the same labels
    lab2 = gbk.nprobe_labels(ix, xq, gt=torch.from_numpy(gt).cuda(), n_classes=C, k=k,
                             kprime=kprime)
    assert torch.equal(lab, lab2)


def test_nprobe_mlp_train_in_library(gbk):
    ix, x, xq, cen = _build(gbk, keep=True)
    xt = torch.from_numpy(datagen.mixture_points(cen, 520, 8192)).cuda()
    losses = []
    params = []
    for _ in range(2):
        net = gbk.MLP(64 + 64, 256, 256, 9, seed=521)
        losses.append(gbk.nprobe_mlp_train(ix, net, xt, epochs=6, batch=1024, seed=522))
        params.append(net.params())
    assert np.all(np.isfinite(losses[0])) and losses[0][-1] < losses[0][0]
    np.testing.assert_array_equal(losses[0], losses[1])  # seeded: bit-reproducible
    assert torch.equal(params[0], params[1])
    # the trained network routes a batch (nprobe = 2^class, capped)
    kq = torch.full((xq.shape[0],), 10, dtype=torch.int32, device="cuda")
    _, _, _, used = gbk.ivfpq_search_batched(ix, xq, kq, 10, None, 64, mlp=net)
    u = used.cpu().numpy()
    assert np.all((u >= 1) & (u <= 64) & ((u & (u - 1)) == 0))


def test_mlp_seeded_init(gbk):
    a = gbk.MLP(192, 256, 256, 9, seed=7).params().cpu().numpy()
    b = gbk.MLP(192, 256, 256, 9, seed=7).params().cpu().numpy()
    c = gbk.MLP(192, 256, 256, 9, seed=8).params().cpu().numpy()
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    w1 = a[:256 * 192]
    assert np.abs(w1).max() <= 1 / np.sqrt(192) and np.abs(w1).max() > 0.9 / np.sqrt(192)
    w3 = a[-(9 * 256 + 9):]
    assert np.abs(w3).max() <= 1 / np.sqrt(256)
    assert abs(w1.mean()) < 0.01 / np.sqrt(192) * 10
