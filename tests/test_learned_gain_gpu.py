"""What the learned nprobe gains over a fixed nprobe, on data whose query difficulty varies.

Queries of two kinds: "easy" ones next to one mixture centre (their neighbours all live in
one inverted list) and "hard" ones midway between two centres (neighbours split over two
lists).  The network is trained by the library's kernels on labels from exact search (the
smallest nprobe in {1, 2, 4, 8, 16} whose 10-R@10 reaches the query's saturated recall);
routed by it, the evaluation queries must reach the recall of the cheapest fixed nprobe that
matches them while probing clearly fewer lists on average."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_1702_08734_gb300 import datagen

pytestmark = pytest.mark.gpu
D, NLIST, TAUS = 32, 64, (1, 2, 4, 8, 16)


def _queries(cen, seed, n):
    """Half easy (centre + 0.3 N(0, I)), half hard (midpoint of two centres + 0.3 N(0, I))."""
    a = datagen.randint(seed, 0, n, NLIST)
    b = (a + 1 + datagen.randint(seed, 0, n, NLIST - 1, stream=1)) % NLIST
    noise = 0.3 * datagen.gaussian_matrix(seed + 1, n, D)
    hard = np.arange(n) % 2 == 1
    q = cen[a].copy()
    q[hard] = 0.5 * (cen[a[hard]] + cen[b[hard]])
    return (q + noise).astype(np.float32)


def _recall(gbk, I, Igt):
    c = torch.empty(I.shape[0], dtype=torch.int32, device="cuda")
    gbk.recall_counts(I.contiguous(), Igt.contiguous(), c)
    return c


def test_learned_nprobe_probes_fewer_lists_at_equal_recall(gbk):
    cen = datagen.mixture_centres(130, NLIST, D, std=5.0)
    xb = torch.from_numpy(datagen.mixture_points(cen, 131, 60000)).cuda()
    ix = gbk.IVFPQIndex(D, NLIST, 8)
    ix.train(xb[:20000], niter=8, coarse_init=datagen.permutation_prefix(132, 20000, NLIST),
             pq_init=datagen.permutation_prefix(133, 20000, 256))
    ix.add(xb)
    coarse = torch.from_numpy(ix.export()["coarse"]).cuda()

    def features_labels(seed, n):
        xq = torch.from_numpy(_queries(cen, seed, n)).cuda()
        _, Igt = gbk.knn_brute(xq, xb, 10)
        rec = torch.stack([_recall(gbk, ix.search(xq, 10, t)[1], Igt) for t in TAUS], 1)
        y = torch.argmax((rec >= rec[:, -1:]).to(torch.int32), dim=1).to(torch.int32)
        clD, _ = gbk.knn_brute(xq, coarse, 64)
        return xq, Igt, gbk.nprobe_features(xq, clD), y

    _, _, F, y = features_labels(134, 8192)
    hist = torch.bincount(y.long(), minlength=len(TAUS)).cpu().numpy()
    assert hist[0] > 2000 and hist[1:].sum() > 2000  # both kinds present in the labels
    sizes = (D + 64, 128, 128, len(TAUS))
    n = sizes[1] * sizes[0] + sizes[1] + sizes[2] * sizes[1] + sizes[2] + sizes[3] * sizes[2] + sizes[3]
    p = omlp.init_params(sizes, datagen.uniform24(135, 0, n).astype(np.float64))
    net = gbk.MLP(*sizes, params=np.concatenate([p[k].ravel() for k in omlp.PARAM_NAMES])
                  .astype(np.float32))
    for ep in range(20):
        perm = torch.from_numpy(np.argsort(datagen.hash_u64(136 + ep, 0, F.shape[0]))).cuda()
        for b0 in range(0, F.shape[0], 512):
            idx = perm[b0:b0 + 512]
            net.train_step(F[idx].contiguous(), y[idx].contiguous(), lr=2e-3)

    xq, Igt, _, _ = features_labels(137, 2000)
    fixed = [float(_recall(gbk, ix.search(xq, 10, t)[1], Igt).float().mean()) / 10 for t in TAUS]
    kq = torch.full((xq.shape[0],), 10, dtype=torch.int32, device="cuda")
    _, I, _, used = gbk.ivfpq_search_batched(ix, xq, kq, 10, None, 16, mlp=net)
    r_learned = float(_recall(gbk, I.view(-1, 10), Igt).float().mean()) / 10
    mean_np = float(used.float().mean())
    tau_eq = next(t for t, r in zip(TAUS, fixed) if r >= r_learned - 0.005)
    print("learned: 10-R@10 %.4f at mean nprobe %.3f; fixed nprobe %s: %s; labels %s"
          % (r_learned, mean_np, TAUS, ["%.4f" % r for r in fixed], hist.tolist()))
    # equal recall with clearly fewer probed lists than the cheapest matching fixed nprobe
    assert r_learned >= fixed[0] + 0.05, (r_learned, fixed)
    assert mean_np <= 0.85 * tau_eq, (mean_np, tau_eq, r_learned, fixed)
