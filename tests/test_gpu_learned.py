"""Learned sub-domain proposal through the C ABI: training gradients against the FP64 oracle, tensor-core
inference against a reference taken in the kernel's precision, trace export, training, and hits of the
learned traversal bit-identical to the plain traversal."""
import os
import tempfile

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_1811_03510_gb300 import ccs, scenegen as sg
from parity import MISS, compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
RNG = np.random.default_rng(77)


@pytest.fixture(scope="module", autouse=True)
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_03510_gb300 import build_ext
    build_ext.build()
    oracle.build()
    torch.cuda.set_device(0)


def _cuda(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def test_gradient_matches_fp64_oracle():
    p = ccs.ccs_proposal_create(seed=3)
    theta = ccs.ccs_proposal_get_params(p).astype(np.float64)
    B = 3000
    X = RNG.normal(size=(B, 24)).astype(np.float32)
    y = RNG.integers(0, 64, size=B).astype(np.uint8)
    grad = torch.zeros(ccs.CCS_PROPOSAL_PARAMS, device="cuda")
    loss = torch.zeros(1, device="cuda")
    ccs.ccs_proposal_grad(p, _cuda(X, np.float32), _cuda(y, np.uint8), B, grad, loss)
    torch.cuda.synchronize()
    L_ref, g_ref = mlp.loss_and_grad(theta, X.astype(np.float64), y)
    assert abs(loss.item() - L_ref) <= 1e-5 * abs(L_ref)
    g = grad.cpu().numpy().astype(np.float64)
    for part, ref in zip(mlp.unpack(g), mlp.unpack(g_ref)):
        rel = np.linalg.norm(part - ref) / max(np.linalg.norm(ref), 1e-30)
        cos = float(part.ravel() @ ref.ravel()) / (np.linalg.norm(part) * np.linalg.norm(ref) + 1e-30)
        assert rel <= 1e-4 and cos > 0.99999, (rel, cos)
    ccs.ccs_proposal_destroy(p)


def test_tensor_core_inference_matches_reference_in_kernel_precision():
    p = ccs.ccs_proposal_create(seed=5)
    theta = ccs.ccs_proposal_get_params(p).astype(np.float64)
    n = 1000   # not a multiple of 32: ragged last warp
    X = RNG.normal(size=(n, 24)).astype(np.float32)
    logits = torch.zeros(n, 64, device="cuda")
    cells = torch.zeros(n, dtype=torch.uint8, device="cuda")
    pmax = torch.zeros(n, device="cuda")
    ccs.ccs_proposal_infer(p, _cuda(X, np.float32), n, logits, cells, pmax)
    torch.cuda.synchronize()
    ref = mlp.forward_bf16(theta, X)
    lg = logits.cpu().numpy().astype(np.float64)
    scale = np.abs(ref).max()
    assert np.abs(lg - ref).max() <= 2e-3 * scale
    c = cells.cpu().numpy()
    top2 = np.sort(ref, axis=1)[:, -2:]
    clear = (top2[:, 1] - top2[:, 0]) > 1e-2 * scale
    assert (c[clear] == ref[clear].argmax(1)).all()
    assert clear.mean() > 0.5
    # where the top two are close, the chosen cell is still a maximum within the logit tolerance
    assert (ref[np.arange(n), c] >= ref.max(1) - 4e-3 * scale).all()
    e = np.exp(ref - ref.max(1, keepdims=True))
    np.testing.assert_allclose(pmax.cpu().numpy(), 1 / e.sum(1), rtol=5e-3)
    ccs.ccs_proposal_destroy(p)


def _root_interval(g, greg, o, d):
    pts = g if greg else g[:16]
    lo, hi = pts.min(0), pts.max(0)
    with np.errstate(divide="ignore", invalid="ignore"):
        ta, tb = (lo - o) / d, (hi - o) / d
    return np.minimum(ta, tb).max(), np.maximum(ta, tb).min()


def _features(g, greg, o, d, t0, t1):
    """The 24 pair features as the library header defines them."""
    an = 0.5 * ((g if greg else g[:16]).min(0) + (g if greg else g[:16]).max(0))
    c = np.array([g[0], g[3], g[12], g[15]]) - an
    S = np.linalg.norm(c, axis=1).max()
    du = d / np.linalg.norm(d)
    f = np.zeros(24)
    f[0:3] = ((o - an) + t0 * np.linalg.norm(d) * du) / S
    f[3:6] = du
    f[6:18] = (c / S).reshape(-1)
    n = np.cross(c[3] - c[0], c[2] - c[1])
    n /= np.linalg.norm(n)
    f[18:21] = n
    f[21] = min((t1 - t0) * np.linalg.norm(d) / S, 4.0)
    f[22] = du @ n
    f[23] = float(greg)
    return f


def test_trace_export_features_and_labels():
    s = sg.config_scene(1)
    for p in (0, int(np.nonzero(s.types == 1)[0][0])):
        P1, t1 = s.P[p:p + 1], s.types[p:p + 1]
        c = P1[0].mean(0)
        r = sg.random_rays(3000, seed=p + 40, radius=2.0)
        r = sg.Rays(r.o, (c[None] + 0.04 * RNG.normal(size=(3000, 3)) - r.o).astype(np.float32), r.tmin, r.tmax)
        sc = ccs.Scene(P1, t1)
        rays = ccs.rays_to_device(r.soa())
        hits = ccs.alloc_hits(r.n)
        feat = torch.zeros(r.n, 24, device="cuda")
        lab = torch.zeros(r.n, dtype=torch.uint8, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        ccs.ccs_trace_export(sc.handle, rays, r.n, hits, ccs.make_opts(), feat, lab, r.n, cnt)
        torch.cuda.synchronize()
        g = ccs.hits_to_numpy(hits)
        hit = np.nonzero(g["pid"] != MISS)[0]
        k = int(cnt.item())
        assert k == len(hit) > 500
        F, Lb = feat.cpu().numpy()[:k], lab.cpu().numpy()[:k]
        # every exported row is the feature vector of one hit ray (order is atomic): match by direction
        dirs = r.d[hit].astype(np.float64)
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        used = set()
        for row, label in zip(F, Lb):
            j = int(np.argmin(np.linalg.norm(dirs - row[3:6].astype(np.float64), axis=1)))
            assert j not in used
            used.add(j)
            i = hit[j]
            o, d = r.o[i].astype(np.float64), r.d[i].astype(np.float64)
            a, b = _root_interval(P1[0].astype(np.float64), bool(t1[0]), o, d)
            f_ref = _features(P1[0].astype(np.float64), bool(t1[0]), o, d, a, b)
            cu, cv = int(round(g["u"][i] * 256 - 0.5)), int(round(g["v"][i] * 256 - 0.5))
            np.testing.assert_allclose(row, f_ref, atol=2e-4)
            assert label == (cv >> 5) * 8 + (cu >> 5)
        sc.close()


def test_training_reduces_loss_and_save_load_roundtrip():
    s = sg.config_scene(2, seed=3)
    r = sg.pinhole_rays(640, 360)
    sc = ccs.Scene(s.P, s.types)
    rays = ccs.rays_to_device(r.soa())
    hits = ccs.alloc_hits(r.n)
    cap = 200000
    feat = torch.zeros(cap, 24, device="cuda")
    lab = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    ccs.ccs_trace_export(sc.handle, rays, r.n, hits, ccs.make_opts(), feat, lab, cap, cnt)
    torch.cuda.synchronize()
    n = min(int(cnt.item()), cap)
    assert n > 10000
    p = ccs.ccs_proposal_create(seed=1)
    loss = torch.zeros(1, device="cuda")
    B = 2048
    losses = []
    for step in range(300):
        i0 = (step * B) % (n - B)
        ccs.ccs_proposal_train_step(p, feat[i0:i0 + B], lab[i0:i0 + B], B, 2e-3, loss)
        if step % 50 == 0 or step == 299:
            torch.cuda.synchronize()
            losses.append(loss.item())
    assert losses[-1] < 0.6 * losses[0], losses
    cells = torch.zeros(n, dtype=torch.uint8, device="cuda")
    ccs.ccs_proposal_infer(p, feat[:n], n, None, cells, None)
    torch.cuda.synchronize()
    acc = (cells[:n] == lab[:n]).float().mean().item()
    assert acc > 0.2, acc   # chance is 1/64
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "prop.bin")
        ccs.ccs_proposal_save(p, path)
        q = ccs.ccs_proposal_load(path)
        assert np.array_equal(ccs.ccs_proposal_get_params(q), ccs.ccs_proposal_get_params(p))
        ccs.ccs_proposal_destroy(q)
    ccs.ccs_proposal_destroy(p)
    sc.close()


@pytest.mark.parametrize("which", ["cfg1_primary", "random", "gregory_ring", "cfg2_primary"])
def test_learned_hits_identical_to_plain(which):
    if which == "cfg1_primary":
        s, r = sg.config_scene(1), sg.pinhole_rays(96, 96)
    elif which == "random":
        s, r = sg.config_scene(2), sg.random_rays(40000, seed=3)
    elif which == "gregory_ring":
        s, r = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True), sg.random_rays(30000, seed=4, target=1.0)
    else:
        s, r = sg.config_scene(2), sg.pinhole_rays(480, 270)
    sc = ccs.Scene(s.P, s.types)
    rays = ccs.rays_to_device(r.soa())
    ref = ccs.alloc_hits(r.n)
    ccs.ccs_intersect(sc.handle, rays, r.n, ref, ccs.make_opts())
    p = ccs.ccs_proposal_create(seed=9)   # an untrained network proposes arbitrary cells: a hard case
    orc = oracle.intersect(s.P, s.types, r.soa(), L=8, flags=True)
    for conf in (0.0, 0.05):
        out = ccs.alloc_hits(r.n)
        ccs.ccs_intersect_learned(sc.handle, p, rays, r.n, out, ccs.make_opts(), conf)
        torch.cuda.synchronize()
        assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
        for a, b in zip(ref, out):
            assert torch.equal(a, b)
        compare(ccs.hits_to_numpy(out), orc, 8)   # the learned traversal against the oracle itself
    ccs.ccs_proposal_destroy(p)
    sc.close()


def _splits(sc, planes, learned=None):
    n = len(planes[0])
    rays = ccs.rays_to_device(planes)
    hits = ccs.alloc_hits(n)
    c = torch.zeros(ccs.CCS_NUM_COUNTERS, dtype=torch.int64, device="cuda")
    if learned is None:
        ccs.ccs_intersect(sc.handle, rays, n, hits, ccs.make_opts(counters=c))
    else:
        ccs.ccs_intersect_learned(sc.handle, learned, rays, n, hits, ccs.make_opts(counters=c), 0.0)
    torch.cuda.synchronize()
    assert ccs.ccs_scene_sync_status(sc.handle) == ccs.CCS_OK
    return int(c[1] + c[2]), ccs.hits_to_numpy(hits)


@pytest.mark.parametrize("local", [False, True])
def test_seeded_best_distance_bounds_what_any_proposal_can_save(local):
    """The most a proposal can save: the search started with the final best distance already known (tmax
    set to the oracle's hit distance, which the inclusive tmax keeps).  Nodes entered before that distance
    must be searched whatever the order, so the seeded run does the least subdivision work any traversal
    can.  On the 1536-patch scene it saves under 3% of the plain traversal's splits on primary rays and
    none on diffuse rays: the closer-first order with sibling pruning already finds the best leaf first.
    The learned traversal, whose proposal is only a depth-3 cell, does more work than the seeded run."""
    s = sg.config_scene(2)
    r = sg.pinhole_rays(480, 270)
    sc = ccs.Scene(s.P, s.types, local=local)
    o = oracle.intersect(s.P, s.types, r.soa(), L=8, local=local)
    hit = o["pid"] != MISS
    seeded = r.soa()
    seeded[7] = np.where(hit, o["t"] * (1 + 1e-6), np.inf).astype(np.float32)
    plain, hp = _splits(sc, r.soa())
    best, hs = _splits(sc, seeded)
    assert np.array_equal(hs["pid"], hp["pid"]) and np.array_equal(hs["t"], hp["t"])
    assert best <= plain < 1.03 * best, (plain, best)
    p = ccs.ccs_proposal_create(seed=9)
    learned, _ = _splits(sc, r.soa(), learned=p)
    assert learned >= best
    ccs.ccs_proposal_destroy(p)
    # diffuse rays leave the (near-convex) sphere: nothing to save
    from oracle.raygen import diffuse_rays
    d = diffuse_rays(s.P, s.types, r.soa(), o, seed=1)
    act = d[7] >= d[6]
    dr = [np.ascontiguousarray(a[act]) for a in d]
    od = oracle.intersect(s.P, s.types, dr, L=8, local=local)
    ds = list(dr)
    ds[7] = np.where(od["pid"] != MISS, od["t"] * (1 + 1e-6), dr[7]).astype(np.float32)
    plain_d, _ = _splits(sc, dr)
    best_d, _ = _splits(sc, ds)
    assert best_d <= plain_d <= 1.03 * best_d + 10, (plain_d, best_d)
    sc.close()
