"""Batching form: pairs of uneven grid and band advanced together (persistent
sweep kernels over a (pair, tile) work queue, PCG iterations replayed from a
CUDA graph, autotuned tile length).  Each pair's arithmetic equals a single
plan's, so gradients, Hessian-vector products and whole registrations must be
bit-identical to per-pair calls: on six small pairs, and on the 64-pair
workload (grids 64^3 to 160x192x160, bands 16^3 to 32^3) with one pair of every
grid size rerun alone.  Batched pairs are also compared with the FP64 oracle
directly (gradient, HVP and a short registration)."""

import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1807_05117_gb300 import synth  # noqa: E402

SHAPES = [((40, 36, 52), (8, 6, 10)), ((32, 32, 32), (8, 8, 8)), ((24, 20, 28), (6, 4, 8)),
          ((16, 24, 20), (4, 6, 4)), ((48, 40, 32), (12, 8, 8)), ((20, 20, 20), (4, 4, 4))]
NT = 6


@pytest.fixture(scope="module")
def setup():
    from paper_1807_05117_gb300 import blr
    pairs = []
    for i, (n, band) in enumerate(SHAPES):
        I0, I1, _ = synth.blob_pair(n, 900 + i, max_disp=2.0)
        vt = synth.random_coefficients(band, 950 + i, 3.0)
        dv = synth.random_direction(band, 970 + i)
        (I0f, _), (I1f, _), (vtf, _), (dvf, _) = synth.as_device_inputs(I0, I1, vt, dv)
        pairs.append(dict(n=n, band=band, I0=torch.from_numpy(I0f).cuda(),
                          I1=torch.from_numpy(I1f).cuda(), vt=torch.from_numpy(vtf).cuda(),
                          dv=torch.from_numpy(dvf).cuda()))
    batch = blr.Batch([(p["n"], p["band"]) for p in pairs], NT)
    for i, p in enumerate(pairs):
        batch.set_images(i, p["I0"], p["I1"])
    plans = []
    for p in pairs:
        pl = blr.Plan(p["n"], p["band"], NT)
        pl.set_images(p["I0"], p["I1"])
        plans.append(pl)
    return blr, pairs, batch, plans


def test_batched_gradient_and_hessvec_equal_single_plans(setup):
    blr, pairs, batch, plans = setup
    gb = [torch.empty_like(p["vt"]) for p in pairs]
    batch.gradient([p["vt"] for p in pairs], gb)
    hb = [torch.empty_like(p["vt"]) for p in pairs]
    batch.hessvec([p["dv"] for p in pairs], hb)
    for p, pl, g, h in zip(pairs, plans, gb, hb):
        gs, hs = torch.empty_like(g), torch.empty_like(h)
        pl.gradient(p["vt"], gs)
        pl.hessvec(p["dv"], hs)
        assert pl.status() == blr.BLR_OK
        assert torch.equal(g, gs)
        assert torch.equal(h, hs)


@pytest.mark.parametrize("forcing", [-1.0, 0.0], ids=["superlinear-eta", "fixed-work"])
def test_batched_newton_equals_single_plans(setup, forcing):
    blr, pairs, batch, plans = setup
    vb = [torch.zeros_like(p["vt"]) for p in pairs]
    reps = batch.newton(vb, 3, 6, 1e-6, forcing)
    for p, pl, v, r in zip(pairs, plans, vb, reps):
        vs = torch.zeros_like(v)
        rs = pl.newton(vs, 3, 6, 1e-6, forcing)
        assert r.status == rs.status == blr.BLR_OK
        assert (r.newton_iters, r.pcg_iters, r.n_hessvec, r.n_halvings) == \
            (rs.newton_iters, rs.pcg_iters, rs.n_hessvec, rs.n_halvings)
        assert r.energy == rs.energy and r.energy0 == rs.energy0
        assert torch.equal(v, vs)
        assert r.energy < r.energy0


def _compare_with_single_plans(blr, pairs, batch, plans):
    gb = [torch.empty_like(p["vt"]) for p in pairs]
    batch.gradient([p["vt"] for p in pairs], gb)
    hb = [torch.empty_like(p["vt"]) for p in pairs]
    batch.hessvec([p["dv"] for p in pairs], hb)
    vb = [torch.zeros_like(p["vt"]) for p in pairs]
    reps = batch.newton(vb, 2, 5, 1e-6, 0.0)
    for p, pl, g, h, v, r in zip(pairs, plans, gb, hb, vb, reps):
        gs, hs = torch.empty_like(g), torch.empty_like(h)
        pl.gradient(p["vt"], gs)
        pl.hessvec(p["dv"], hs)
        assert torch.equal(g, gs)
        assert torch.equal(h, hs)
        vs = torch.zeros_like(v)
        rs = pl.newton(vs, 2, 5, 1e-6, 0.0)
        assert r.status == rs.status == blr.BLR_OK
        assert (r.newton_iters, r.pcg_iters, r.n_halvings) == \
            (rs.newton_iters, rs.pcg_iters, rs.n_halvings)
        assert r.energy == rs.energy
        assert torch.equal(v, vs)


@pytest.mark.parametrize("useg,gather", [(1, 1), (1, 0), (0, 0)],
                         ids=["kept-gradients-gather", "kept-gradients-march", "interpolated"])
def test_both_gradient_choices_equal_single_plans(setup, useg, gather):
    """Batched sweeps that read the kept state gradients (with the incremental
    steps in the gather or the march form) and ones that interpolate grad m^n
    give the single plans' results bit for bit."""
    blr, pairs, batch, plans = setup
    tun = batch.tuning()
    assert tun["kept_gradients"] == 1
    batch.set_tuning(use_kept_gradients=useg, incremental_gather=gather)
    assert (batch.tuning()["use_kept_gradients"], batch.tuning()["incremental_gather"]) == (useg, gather)
    try:
        if useg != tun["use_kept_gradients"]:
            with pytest.raises(blr.BlrError):   # the change dropped the current points
                batch.hessvec([p["dv"] for p in pairs], [torch.empty_like(p["vt"]) for p in pairs])
        _compare_with_single_plans(blr, pairs, batch, plans)
    finally:
        batch.set_tuning(use_kept_gradients=tun["use_kept_gradients"],
                         incremental_gather=tun["incremental_gather"])
    with pytest.raises(blr.BlrError):
        batch.set_tuning(kept_gradients=0)


@pytest.mark.parametrize("solo_min", [30000, 1], ids=["three-solo", "all-solo"])
def test_solo_pairs_equal_single_plans(setup, solo_min):
    """Pairs that run solo (their own plans' tuned kernels, their own PCG graphs)
    beside queued pairs, and a batch of solo pairs only, give the single plans'
    results bit for bit."""
    blr, pairs, batch, plans = setup
    tun = batch.tuning()
    batch.set_tuning(solo_min_voxels=solo_min)
    want = sum(1 for p in pairs if p["n"][0] * p["n"][1] * p["n"][2] >= solo_min)
    assert batch.tuning()["solo_pairs"] == want
    try:
        _compare_with_single_plans(blr, pairs, batch, plans)
    finally:
        batch.set_tuning(solo_min_voxels=tun["solo_min_voxels"])
    assert batch.tuning()["solo_pairs"] == tun["solo_pairs"]


def test_batch_rejects_mixed_shapes_of_time(setup):
    blr = setup[0]
    with pytest.raises(blr.BlrError) as ei:
        blr.Batch([blr.make_params((16, 16, 16), (4, 4, 4), 4),
                   blr.make_params((16, 16, 16), (4, 4, 4), 5)])
    assert ei.value.code == blr.BLR_EINVAL


# --- the many-pair workload: 64 pairs, grids {64^3 .. 160x192x160}, bands
# {16^3, 24^3, 32^3}, 3-8 voxel phantom warps, 10 Newton x <= 20 PCG ---------------


@pytest.mark.slow
def test_uneven_batch_of_64_pairs():
    import multiprocessing as mp
    from paper_1807_05117_gb300 import blr
    pairs = synth.uneven_pairs(64, 4)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        imgs = pool.starmap(synth.phantom_pair_f32,
                            [(p["n"], p["seed"], p["max_disp"]) for p in pairs])
    batch = blr.Batch([(p["n"], p["band"]) for p in pairs], 10)
    for i, (I0, I1) in enumerate(imgs):
        batch.set_images(i, torch.from_numpy(I0).cuda(), torch.from_numpy(I1).cuda())
    vb = [torch.zeros((3,) + p["band"], dtype=torch.complex64, device="cuda") for p in pairs]
    reps = batch.newton(vb, 10, 20, 1e-2)
    for r in reps:
        assert r.status == blr.BLR_OK
        assert r.energy < r.energy0
    # one pair of every grid size against its own single plan, bit for bit
    chosen = {}
    for i, p in enumerate(pairs):
        chosen.setdefault(p["n"], i)
    for i in chosen.values():
        p = pairs[i]
        pl = blr.Plan(p["n"], p["band"], 10)
        pl.set_images(torch.from_numpy(imgs[i][0]).cuda(), torch.from_numpy(imgs[i][1]).cuda())
        vs = torch.zeros_like(vb[i])
        rs = pl.newton(vs, 10, 20, 1e-2)
        assert (reps[i].newton_iters, reps[i].pcg_iters, reps[i].n_halvings) == \
            (rs.newton_iters, rs.pcg_iters, rs.n_halvings)
        assert reps[i].energy == rs.energy
        assert torch.equal(vb[i], vs)
        pl.close()
    batch.close()


# --- batched pairs against the FP64 oracle ------------------------------------
# Shapes of the many-pair workload (the largest grid with band 24^3, 96^3 with
# band 16^3, 64^3 with band 32^3 and 128^3 with band 24^3): the batched gradient
# and Gauss-Newton HVP of each pair within the FP32 bounds of the single-plan
# parity tests (relative L2 1e-4), so a fault shared by the batched and the
# single-plan code (tile tails of these grids, their bands) cannot pass.

# coefficient bounds give 0.56-0.64 voxel per step (both cell choices, all 27
# transpose neighbours)
ORACLE_PAIRS = [((160, 192, 160), (24, 24, 24), 95.0), ((96, 96, 96), (16, 16, 16), 62.0),
                ((64, 64, 64), (32, 32, 32), 120.0), ((128, 128, 128), (24, 24, 24), 100.0)]


@pytest.mark.slow
def test_batched_pairs_match_the_oracle():
    from oracle import blr_oracle as O
    from paper_1807_05117_gb300 import blr
    nt = 10
    data = []
    for i, (n, band, bound) in enumerate(ORACLE_PAIRS):
        I0, I1, _ = synth.phantom_pair(n, 5100 + i, max_disp=5.0)
        vt = synth.random_coefficients(band, 5200 + i, bound=bound)
        dv = synth.random_direction(band, 5300 + i)
        data.append(synth.as_device_inputs(I0, I1, vt, dv))
    batch = blr.Batch([(n, band) for n, band, _ in ORACLE_PAIRS], nt)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    for i, ((I0f, _), (I1f, _), _, _) in enumerate(data):
        batch.set_images(i, dev(I0f), dev(I1f))
    vts = [dev(d[2][0]) for d in data]
    dvs = [dev(d[3][0]) for d in data]
    gb = [torch.empty_like(v) for v in vts]
    hb = [torch.empty_like(v) for v in vts]
    batch.gradient(vts, gb)
    batch.hessvec(dvs, hb)
    torch.cuda.synchronize()
    batch.close()
    for (n, band, _), d, g, h in zip(ORACLE_PAIRS, data, gb, hb):
        (_, I0d), (_, I1d), (_, vtd), (_, dvd) = d
        pt = O.Point(vtd, I0d, I1d, O.Params(n, band, nt))
        assert pt.cfl < 1.0
        g_ref = pt.gradient()[0]
        h_ref = pt.gn_hessvec(dvd)[0]
        eg = np.linalg.norm(g.cpu().numpy() - g_ref) / np.linalg.norm(g_ref)
        eh = np.linalg.norm(h.cpu().numpy() - h_ref) / np.linalg.norm(h_ref)
        assert eg <= 1e-4 and eh <= 1e-4, (n, band, eg, eh)


def test_batched_newton_matches_the_oracle():
    """Two small uneven pairs (16^3 / band 4^3, 24x20x16 / band 6^3), 3 Newton
    updates each: Newton counts equal, final energy within 1e-3, PCG totals
    within +-1 per update (the single-plan registration bars)."""
    from oracle import blr_oracle as O
    from paper_1807_05117_gb300 import blr
    shapes, nt = [((16, 16, 16), (4, 4, 4)), ((24, 20, 16), (6, 6, 6))], 4
    batch = blr.Batch(shapes, nt)
    refs, vts = [], []
    for i, (n, band) in enumerate(shapes):
        I0, I1, _ = synth.blob_pair(n, 5400 + i, max_disp=2.0)
        (I0f, I0d), (I1f, I1d) = synth.as_device_inputs(I0, I1)
        batch.set_images(i, torch.from_numpy(I0f).cuda(), torch.from_numpy(I1f).cuda())
        vts.append(torch.zeros((3,) + band, dtype=torch.complex64, device="cuda"))
        refs.append(O.newton(np.zeros((3,) + band, complex), I0d, I1d, O.Params(n, band, nt),
                             max_newton=3, max_pcg=6, gtol=1e-6))
    reps = batch.newton(vts, 3, 6, 1e-6)
    batch.close()
    for r, ref in zip(reps, refs):
        assert r.status == blr.BLR_OK
        assert r.newton_iters == ref.iterations
        assert abs(r.energy0 - ref.energies[0]) <= 1e-5 * ref.energies[0]
        assert abs(r.energy - ref.energies[-1]) <= 1e-3 * ref.energies[-1]
        assert abs(r.pcg_iters - sum(ref.pcg_iterations)) <= ref.iterations
