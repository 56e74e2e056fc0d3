"""Densification under consensus on the GPU against the FP64 oracle
(decisions bit-exact wherever the oracle's decision margin is at least 1e-6,
the rest counted; offsets and emitted parameters within the parity bar), and
in the trainer: the rebuilt layout keeps every invariant of the consensus and
training goes on."""
import numpy as np
import pytest
import torch

from paper_2405_13943_b300 import synth as S

pytestmark = pytest.mark.gpu
REL = 1e-3


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_13943_b300 import build as B
    B.build()
    from oracle import oracle as O
    from paper_2405_13943_b300 import dogs, serve, trainer
    return dogs, O, serve, trainer


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def problem(seed, n_pts=4000, deg=1):
    rng = np.random.default_rng(seed)
    xy = rng.uniform(0, 100, (n_pts, 2))
    split, order = S.block_split(xy, 2, 2, [0.3, 0.2, 0.35, 0.15], 0.1)
    z = S.cube_scene(n_pts, seed, sh_degree=deg).subset(order)
    # spread the decisions: opacity logits around logit(0.005), log-scales around log(0.01)
    z.opacity_logits[:] = rng.normal(-5.3, 1.0, n_pts).astype(np.float32)
    z.log_scales[:] = rng.normal(np.log(0.01), 0.7, (n_pts, 3)).astype(np.float32)
    stats = np.empty(2 * split.n_copies, np.float32)
    stats[1::2] = rng.integers(0, 4, split.n_copies).astype(np.float32)
    stats[0::2] = (stats[1::2] * rng.uniform(0, 4e-4, split.n_copies)).astype(np.float32)
    return split, z, stats


def test_statistic_matches_oracle(mods):
    D, O, _, _ = mods
    cams = [S.cube_camera(64, 48), S.cube_camera(40, 40)]
    cams[1].block = 1
    vb = D.ViewBatch(cams, [0, 300, 500], 16, 16)
    rng = np.random.default_rng(3)
    n_rec = vb.n_rec
    rect = np.zeros((n_rec, 2), np.uint32)
    kept = rng.random(n_rec) < 0.6
    rect[kept, 1] = 1 | (1 << 16)                      # a one-tile rectangle [0,1) x [0,1)
    drec = rng.normal(0, 1e-3, (n_rec, 12)).astype(np.float32)
    vb.rect.copy_(torch.from_numpy(rect.view(np.int32).reshape(-1)))
    vb.drec.copy_(torch.from_numpy(drec.reshape(-1)))
    stats = torch.zeros(2 * 500, dtype=torch.float32, device="cuda")
    for _ in range(2):                                  # two iterations accumulate
        D.dg_densify_stats(vb, stats)
    torch.cuda.synchronize()
    owner = np.concatenate([np.arange(0, 300), np.arange(300, 500)])
    wh = np.array([[64, 48]] * 300 + [[40, 40]] * 200)
    s, c = O.densify_stats(kept, drec[:, :2], wh, owner, 500)
    got = stats.cpu().numpy()
    np.testing.assert_allclose(got[0::2], 2 * s, rtol=1e-5, atol=1e-9)
    np.testing.assert_array_equal(got[1::2], 2 * c)


MARGIN = 1e-6          # decisions nearer their threshold than this may differ between FP32 and FP64


@pytest.mark.parametrize("seed", [1, 2])
def test_decisions_match_oracle_outside_margin(mods, seed):
    """The GPU decides in FP32 on FP32 sums; the oracle in FP64.  Every
    decision with a relative margin of at least 1e-6 must agree; the others
    are counted and must stay a negligible share."""
    D, O, _, _ = mods
    split, z, stats = problem(seed)
    zb = D.GaussianBuffer.from_synth(z)
    kw = dict(grad_threshold=2e-4, percent_dense=0.01, extent=1.0, min_opacity=0.005)
    codes, offsets = D.dg_densify_decide(zb, torch.from_numpy(split.g_off).cuda(),
                                         torch.from_numpy(split.g_copies).cuda(), torch.from_numpy(stats).cuda(), **kw)
    torch.cuda.synchronize()
    want, margin = O.densify_decide(O.params_from(z), 1, stats[0::2], stats[1::2], split.g_off, split.g_copies,
                                    return_margin=True, **kw)
    got = codes.cpu().numpy()
    ok = margin >= MARGIN
    assert (~ok).sum() <= max(1, int(1e-4 * z.n))
    np.testing.assert_array_equal(got[ok], want[ok])
    assert len(set(want[ok].tolist())) == 4             # every branch taken
    # the offsets are the exclusive scan of the GPU's own output counts
    counts = np.where(got == O.DENSIFY_PRUNE, 0, np.where(got == O.DENSIFY_KEEP, 1, 2))
    np.testing.assert_array_equal(offsets.cpu().numpy().view(np.uint32), np.concatenate([[0], np.cumsum(counts)]))


def curated(O, split, z, stats, kw):
    """The problem with every near-threshold Gaussian moved clear of its
    thresholds (its statistic zeroed and its opacity raised: a plain keep),
    so that both sides must take every decision alike."""
    for _ in range(3):
        _, margin = O.densify_decide(O.params_from(z), 1, stats[0::2], stats[1::2], split.g_off, split.g_copies,
                                     return_margin=True, **kw)
        near = np.nonzero(margin < MARGIN)[0]
        if near.size == 0:
            return z, stats
        z.opacity_logits[near] = 0.0
        for i in near:
            cps = split.g_copies[split.g_off[i]:split.g_off[i + 1]]
            stats[2 * cps] = 0.0
            stats[2 * cps + 1] = 0.0
    raise AssertionError("near-threshold Gaussians left after curation")


@pytest.mark.parametrize("seed", [1, 2])
def test_offsets_and_emission_match_oracle(mods, seed):
    D, O, _, _ = mods
    kw = dict(grad_threshold=2e-4, percent_dense=0.01, extent=1.0, min_opacity=0.005)
    split, z, stats = problem(seed)
    z, stats = curated(O, split, z, stats, kw)
    zb = D.GaussianBuffer.from_synth(z)
    codes, offsets = D.dg_densify_decide(zb, torch.from_numpy(split.g_off).cuda(),
                                         torch.from_numpy(split.g_copies).cuda(), torch.from_numpy(stats).cuda(), **kw)
    torch.cuda.synchronize()
    oz = O.params_from(z)
    want = O.densify_decide(oz, 1, stats[0::2], stats[1::2], split.g_off, split.g_copies, **kw)
    np.testing.assert_array_equal(codes.cpu().numpy(), want)
    assert len(set(want.tolist())) == 4
    counts = np.where(want == O.DENSIFY_PRUNE, 0, np.where(want == O.DENSIFY_KEEP, 1, 2))
    off = offsets.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(off, np.concatenate([[0], np.cumsum(counts)]))
    # emission from seeded normals
    xi = np.random.default_rng(seed + 100).normal(size=(z.n, 2, 3)).astype(np.float32)
    n_out = int(off[-1])
    zn, src, orig = D.dg_densify_emit(zb, codes, offsets, torch.from_numpy(xi.reshape(-1)).cuda(), n_out)
    torch.cuda.synchronize()
    ozn, osrc, oorig = O.densify_emit(oz, 1, want, xi.astype(np.float64))
    np.testing.assert_array_equal(src.cpu().numpy(), osrc)
    np.testing.assert_array_equal(orig.cpu().numpy().astype(bool), oorig)
    g, w = O.split_params(O.params_from(zn.to_synth()), 1), O.split_params(ozn, 1)
    for name in ("mean", "quat", "scale", "sh", "opacity"):
        assert rel_l2(g[name], w[name]) <= 1e-6, name
    # copied rows are exact
    same = ~np.isin(np.arange(n_out), np.nonzero(want[osrc] == O.DENSIFY_SPLIT)[0])
    np.testing.assert_array_equal(O.params_from(zn.to_synth())[same], ozn[same].astype(np.float32))


def test_gather_rows_leaves_negative_rows(mods):
    D, O, _, _ = mods
    a = D.GaussianBuffer.from_synth(S.cube_scene(50, 4, sh_degree=2))
    b = D.GaussianBuffer.from_synth(S.cube_scene(30, 5, sh_degree=2))
    before = b.to_synth()
    idx = np.where(np.arange(30) % 3 == 0, -1, (np.arange(30) * 7) % 50).astype(np.int32)
    D.dg_gather_rows(a, torch.from_numpy(idx).cuda(), b)
    torch.cuda.synchronize()
    pa, pb, p0 = O.params_from(a.to_synth()), O.params_from(b.to_synth()), O.params_from(before)
    for r in range(30):
        np.testing.assert_array_equal(pb[r], p0[r] if idx[r] < 0 else pa[idx[r]])


@pytest.mark.parametrize("layout", ["inplace", "resort"])
def test_trainer_densifies_under_consensus(mods, layout):
    D, O, srv, T = mods
    from paper_2405_13943_b300 import densify as DZ
    wl = S.dogs_workload(40_000, 2, 2, 0.1, 41, views_per_step=1, pool=2, width=200, height=150)
    z0 = D.GaussianBuffer.from_synth(wl.z0)
    gt = D.GaussianBuffer.from_synth(wl.gt)
    targets = [srv.render_views(gt, vs).image.clone() for vs in wl.views]
    cfg = DZ.DensifyConfig(interval=2, start=2, until=7, grad_threshold=1e-6, min_opacity=0.3, layout=layout)
    tr = T.DogsTrainer(wl.split, z0, wl.views, targets, rho=(1e-2,) * 5, loss="l1", intv=1, densify=cfg)
    tr.calibrate_capacity()
    n0 = tr.z.n
    for _ in range(8):
        tr.step()
        torch.cuda.synchronize()
        assert not tr.overflowed()
    log = tr.densify_log
    assert [e["t"] for e in log] == [2, 4, 6]
    for e in log:
        assert e["after"] == e["keep"] + 2 * (e["clone"] + e["split"])
        assert e["prune"] > 0 and e["clone"] + e["split"] > 0
    assert tr.z.n == log[-1]["after"] and tr.z.n != n0
    sp = tr.split
    # layout invariants: every global held, shared ones first and held by several blocks
    cnt = np.diff(sp.g_off)
    assert (cnt >= 1).all() and tr._shared_first
    assert int(sp.copy_shared().sum()) == int(cnt[cnt > 1].sum())
    # after the consensus of the last iteration the duals of each shared global
    # sum to zero, up to a few ulps of the parameters (positions are ~1e3 m)
    u = O.params_from(tr.u.to_synth())
    zz = O.params_from(tr.z.to_synth())
    tol = 8 * 2.0 ** -23 * np.abs(zz).max(0) + 1e-6
    for i in np.nonzero(cnt > 1)[0][:500]:
        cps = sp.g_copies[sp.g_off[i]:sp.g_off[i + 1]]
        assert (np.abs(u[cps].sum(0)) <= tol).all()
    # unshared copies equal their global after the consensus
    un = np.nonzero(cnt == 1)[0]
    x = O.params_from(tr.x.to_synth())
    z = O.params_from(tr.z.to_synth())
    np.testing.assert_array_equal(x[sp.g_copies[sp.g_off[un]]], z[un])
    assert np.isfinite(tr.vb.loss.cpu().numpy()).all()


def test_checkpoint_after_densification_resumes(mods, tmp_path):
    """A checkpoint taken after a densification carries the new layout and
    the statistics; a trainer built on the run's original layout takes them
    and continues as the original run does."""
    D, O, srv, T = mods
    from paper_2405_13943_b300 import densify as DZ
    wl = S.dogs_workload(30_000, 2, 2, 0.1, 43, views_per_step=1, pool=2, width=160, height=120)
    gt = D.GaussianBuffer.from_synth(wl.gt)
    targets = [srv.render_views(gt, vs).image.clone() for vs in wl.views]
    cfg = DZ.DensifyConfig(interval=2, start=2, until=9, grad_threshold=1e-6, min_opacity=0.3)
    kw = dict(rho=(1e-2,) * 5, loss="l1", intv=1, densify=cfg)
    a = T.DogsTrainer(wl.split, D.GaussianBuffer.from_synth(wl.z0), wl.views, targets, **kw)
    a.calibrate_capacity()
    for _ in range(4):                                  # densifies at t = 2
        a.step()
    p = str(tmp_path / "dens.ckpt")
    a.save_checkpoint(p)
    b = T.DogsTrainer(wl.split, D.GaussianBuffer.from_synth(wl.z0), wl.views, targets, **kw)
    b.load_checkpoint(p)
    torch.cuda.synchronize()
    assert b.t == a.t and b.z.n == a.z.n and b.split.n_copies == a.split.n_copies
    for n in ("z", "x", "u", "m", "v"):
        assert torch.equal(getattr(a, n).data, getattr(b, n).data), n
    assert torch.equal(a.dstats, b.dstats)
    for _ in range(3):                                  # densifies again at t = 4 and 6 on both
        a.step()
        b.step()
    torch.cuda.synchronize()
    assert a.z.n == b.z.n
    ga, gb = O.params_from(a.z.to_synth()), O.params_from(b.z.to_synth())
    assert rel_l2(gb, ga) <= REL


def test_opacity_reset_matches_oracle_and_runs_on_schedule(mods):
    D, O, srv, T = mods
    g = S.cube_scene(3000, 8, sh_degree=1)
    g.opacity_logits[:] = np.random.default_rng(8).normal(-3.0, 2.0, g.n).astype(np.float32)
    gb = D.GaussianBuffer.from_synth(g)
    m, v = gb.like(), gb.like()
    m.data.fill_(1.0)
    v.data.fill_(2.0)
    D.dg_reset_opacity(gb, 0.01, m, v)
    torch.cuda.synchronize()
    want = O.reset_opacity(O.params_from(g), 1, 0.01)
    got = O.params_from(gb.to_synth())
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-6)
    assert (got[:, -1] < want[:, -1] + 1e-6).all() and (g.opacity_logits < np.log(0.01 / 0.99)).any()
    mm = O.params_from(m.to_synth())
    assert (mm[:, -1] == 0).all() and (mm[:, :-1] == 1).all()
    from paper_2405_13943_b300 import densify as DZ
    wl = S.dogs_workload(20_000, 2, 2, 0.1, 47, views_per_step=1, pool=2, width=128, height=96)
    gt = D.GaussianBuffer.from_synth(wl.gt)
    targets = [srv.render_views(gt, vs).image.clone() for vs in wl.views]
    cfg = DZ.DensifyConfig(interval=1000, start=1000, until=100, opacity_reset=3)
    tr = T.DogsTrainer(wl.split, D.GaussianBuffer.from_synth(wl.z0), wl.views, targets, loss="l1", intv=1,
                       densify=cfg)
    tr.calibrate_capacity()
    cap = np.log(0.01 / 0.99)
    for t in range(4):
        tr.step()
        torch.cuda.synchronize()
        zo = O.params_from(tr.z.to_synth())[:, -1]
        if t == 3:
            assert (zo <= cap + 1e-6).all()          # reset after the consensus of iteration 3
        else:
            assert (zo > cap + 1e-3).any()


def inplace_layout_reference(O, split, codes):
    """The densified layout in the old order, written out plainly: block by
    block, every old copy replaced by its Gaussian's outputs (children after
    their parent); a new copy carries the old copy's state when its Gaussian
    is the parent itself; each new global's copies listed in block order."""
    outs = np.where(codes == O.DENSIFY_PRUNE, 0, np.where(codes == O.DENSIFY_KEEP, 1, 2))
    offsets = np.concatenate([[0], np.cumsum(outs)])
    gid, carry, blk_off, blk_nsh = [], [], [0], []
    for k in range(split.K):
        for c in range(split.blk_off[k], split.blk_off[k + 1]):
            if c == split.blk_off[k] + split.blk_nshared[k]:
                blk_nsh.append(len(gid) - blk_off[-1])
            g = split.copy_gid[c]
            for h in range(outs[g]):
                gid.append(offsets[g] + h)
                carry.append(c if h == 0 and codes[g] != O.DENSIFY_SPLIT else -1)
        if len(blk_nsh) == k:
            blk_nsh.append(len(gid) - blk_off[-1])
        blk_off.append(len(gid))
    lists = [[] for _ in range(int(offsets[-1]))]
    for nc, j in enumerate(gid):
        lists[j].append(nc)
    g_off = np.concatenate([[0], np.cumsum([len(l) for l in lists])])
    g_copies = np.array([c for l in lists for c in l], np.int64)
    return (np.array(gid), np.array(carry), np.array(blk_off), np.array(blk_nsh), g_off, g_copies,
            int(offsets[split.n_shared_globals]))


@pytest.mark.parametrize("seed", [3, 4])
def test_inplace_layout_matches_reference(mods, seed):
    D, O, _, _ = mods
    rng = np.random.default_rng(seed)
    n = 5000
    xy = rng.uniform(0, 100, (n, 2))
    split, _ = S.block_split(xy, 2, 3, rng.dirichlet(np.full(6, 2.0)), 0.15)
    codes = rng.choice(4, size=n, p=[0.6, 0.1, 0.2, 0.1]).astype(np.int32)
    outs = np.where(codes == O.DENSIFY_PRUNE, 0, np.where(codes == O.DENSIFY_KEEP, 1, 2))
    offsets = np.concatenate([[0], np.cumsum(outs)]).astype(np.uint32)
    dev = "cuda"
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dt)).to(dev)
    g_off, g_cp, cp_off, gid, carry = None, None, None, None, None
    g_off, g_cp, gid, carry, cp_off = D.dg_densify_layout(t(codes, np.int32), t(offsets.view(np.int32), np.int32),
                                                          t(split.g_off, np.int64), t(split.g_copies, np.int32),
                                                          t(split.copy_gid, np.int32))
    torch.cuda.synchronize()
    w_gid, w_carry, w_blk, w_nsh, w_goff, w_gcp, w_nshg = inplace_layout_reference(O, split, codes)
    np.testing.assert_array_equal(gid.cpu().numpy(), w_gid)
    np.testing.assert_array_equal(carry.cpu().numpy(), w_carry)
    np.testing.assert_array_equal(g_off.cpu().numpy(), w_goff)
    np.testing.assert_array_equal(g_cp.cpu().numpy(), w_gcp)
    co = cp_off.cpu().numpy().view(np.uint32).astype(np.int64)
    np.testing.assert_array_equal(co[split.blk_off], w_blk)
    np.testing.assert_array_equal(co[split.blk_off[:-1] + split.blk_nshared] - co[split.blk_off[:-1]], w_nsh)
    assert int(offsets[split.n_shared_globals]) == w_nshg


def test_histogram_counts_values_in_range(mods):
    D, O, _, _ = mods
    rng = np.random.default_rng(12)
    v = rng.integers(-3, 9, 100_003).astype(np.int32)
    got = D.dg_histogram_i32(torch.from_numpy(v).cuda(), -1, 6)
    want = np.array([(v == b).sum() for b in range(-1, 5)])
    np.testing.assert_array_equal(got, want)
    assert D.dg_histogram_i32(torch.zeros(0, dtype=torch.int32, device="cuda"), 0, 4).sum() == 0
