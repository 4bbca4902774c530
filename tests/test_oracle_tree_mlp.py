"""Pins of the tree-invariant checker and of the float64 regressor reference.

The checker is pinned by a binary radix tree built here top-down from its
definition (Sec. 2.1: each node is an interval of sorted Morton order, split
where the highest differing bit of the index-augmented code changes), which
it must accept, and by planted mistakes, which it must reject.  The regressor
reference is pinned by central finite differences and by torch autograd."""
import numpy as np
import pytest

import datagen
import oracle
from oracle import mlp, tree_check


def _radix_tree_records(prims, key_bits=30):
    """Tree over sorted (code, index) built recursively from the definition."""
    prims = np.asarray(prims, np.float32)
    n = prims.shape[0]
    sb, _ = oracle.scene_box(prims)
    codes = oracle.morton(prims, sb, key_bits)
    perm = np.lexsort((np.arange(n), codes))
    sc = codes[perm]
    boxes = tree_check.prim_boxes(prims)
    W = 64

    def aug(t):  # index-augmented key as a Python int
        return (int(sc[t]) << W) | t

    recs = np.zeros((2 + 2 * max(n - 1, 0), 8), np.float32)
    encv = recs[:, 3].view(np.int32)
    auxv = recs[:, 7].view(np.int32)
    next_id = [1]

    def build(i, j, slot):
        # returns (lo, hi) of node covering sorted positions [i, j], writes its record at slot
        if i == j:
            lo, hi = boxes[perm[i], :3], boxes[perm[i], 3:]
            recs[slot, 0:3] = lo
            recs[slot, 4:7] = hi
            encv[slot] = ~int(perm[i])
            auxv[slot] = 1
            return lo, hi
        node = 0 if slot == 0 else next_id[0]
        if slot != 0:
            next_id[0] += 1
        x = aug(i) ^ aug(j)
        bit = x.bit_length() - 1
        g = i
        while g < j and not ((aug(g + 1) >> bit) & 1):
            g += 1
        llo, lhi = build(i, g, 2 + 2 * node)
        rlo, rhi = build(g + 1, j, 3 + 2 * node)
        lo, hi = np.minimum(llo, rlo), np.maximum(lhi, rhi)
        recs[slot, 0:3] = lo
        recs[slot, 4:7] = hi
        encv[slot] = node
        auxv[slot] = j - i + 1
        return lo, hi

    if n:
        build(0, n - 1, 0)
    return recs, perm, sc, sb


@pytest.mark.parametrize("n", [1, 2, 3, 17, 300])
@pytest.mark.parametrize("dist", ["cube", "dup"])
def test_tree_checker_accepts_definition_tree(n, dist):
    p = datagen.cube(n, 60 + n) if dist == "cube" else np.repeat(datagen.cube((n + 3) // 4, 61), 4, 0)[:n]
    recs, perm, sc, sb = _radix_tree_records(p)
    st = tree_check.check_lbvh(recs, p, perm, sc, sb)
    assert st["n"] == n


def _mutants(recs):
    enc = lambda r: r[:, 3].view(np.int32)
    out = []
    r = recs.copy(); r[5, 0] -= 0.01; out.append(("box grown", r))
    r = recs.copy(); r[0, 4] += 0.5; out.append(("root box", r))
    r = recs.copy(); r[2:4] = r[3:1:-1]; out.append(("children swapped", r))
    r = recs.copy()
    leaves = np.nonzero(enc(r)[2:] < 0)[0] + 2
    enc(r)[leaves[1]] = enc(r)[leaves[0]]; out.append(("leaf duplicated", r))
    r = recs.copy()
    ints = np.nonzero(enc(r)[2:] > 0)[0] + 2
    enc(r)[ints[0]] = 0; out.append(("cycle to root", r))
    aux = lambda r: r[:, 7].view(np.int32)
    r = recs.copy(); aux(r)[ints[1]] += 1; out.append(("leaf count of an internal child", r))
    r = recs.copy(); aux(r)[leaves[2]] = 0; out.append(("leaf count of a leaf", r))
    r = recs.copy(); aux(r)[0] -= 1; out.append(("leaf count of the root", r))
    return out


@pytest.mark.parametrize("which", range(8))
def test_tree_checker_rejects_planted_mistakes(which):
    p = datagen.cube(64, 62)
    recs, perm, sc, sb = _radix_tree_records(p)
    name, bad = _mutants(recs)[which]
    with pytest.raises(tree_check.TreeError):
        tree_check.check_lbvh(bad, p, perm, sc, None)


def test_tree_checker_rejects_wrong_split_and_bad_sort():
    p = datagen.cube(40, 63)
    recs, perm, sc, sb = _radix_tree_records(p)
    with pytest.raises(tree_check.TreeError):
        tree_check.check_lbvh(recs, p, perm[::-1].copy(), sc, sb)
    # split moved by one position: swap the last leaf of a left subtree into the right one
    # (keeps a valid-looking tree but breaks the highest-differing-bit split)
    sc2 = sc.copy()
    sc2[:] = 7  # all codes equal: splits must then follow the index bits only
    with pytest.raises(tree_check.TreeError):
        tree_check.check_lbvh(recs, p, perm, sc2, sb)


# ------------------------------------------------------------------ MLP

def _rand_theta(seed=0):
    return mlp.he_init(np.random.default_rng(seed)) + 0.01 * np.random.default_rng(seed + 1).standard_normal(mlp.N_PARAMS)


def test_param_count():
    assert mlp.N_PARAMS == 3 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 4481


def test_backward_matches_central_differences():
    g = np.random.default_rng(70)
    theta = _rand_theta(70)
    x = g.random((16, 3))
    t = g.standard_normal(16)
    _, grad = mlp.backward(theta, x, t)
    h = 1e-6
    idx = g.choice(mlp.N_PARAMS, 120, replace=False)
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (mlp.loss(theta + e, x, t) - mlp.loss(theta - e, x, t)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(grad[i])) + 1e-8, (i, fd, grad[i])


def test_forward_backward_match_torch_autograd():
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(71)
    theta = _rand_theta(71)
    x = g.random((33, 3))
    t = g.standard_normal(33)
    p = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in mlp.unpack(theta.copy()).items()}
    X = torch.tensor(x)
    h1 = torch.relu(torch.nn.functional.linear(X, p["W1"], p["b1"]))
    h2 = torch.relu(torch.nn.functional.linear(h1, p["W2"], p["b2"]))
    y = h2 @ p["w3"] + p["b3"]
    L = torch.mean((y - torch.tensor(t)) ** 2)
    L.backward()
    y_or, _ = mlp.forward(theta, x)
    assert np.allclose(y_or, y.detach().numpy(), rtol=1e-12, atol=1e-12)
    loss, grad = mlp.backward(theta, x, t)
    assert abs(loss - L.item()) <= 1e-12 * max(1, abs(loss))
    tg = np.concatenate([p[k].grad.numpy().ravel() for k, _ in mlp.SIZES])
    assert np.allclose(grad, tg, rtol=1e-10, atol=1e-12)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(72)
    theta = _rand_theta(72)
    w = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([w], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    ad = mlp.Adam(mlp.N_PARAMS)
    th = theta.copy()
    for _ in range(5):
        grad = g.standard_normal(mlp.N_PARAMS)
        w.grad = torch.tensor(grad)
        opt.step()
        th = ad.step(th, grad)
    assert np.allclose(th, w.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_normalise_and_label():
    sb = np.array([0, 1, 2, 1, 1, 4], np.float32)
    x = mlp.normalise(np.array([[0.5, 1, 3]]), sb)
    assert x.tolist() == [[0.5, 0.0, 0.5]]
    assert np.allclose(mlp.label(np.array([4.0, 0.0])), [np.log(2.0), np.log(1e-30)])
