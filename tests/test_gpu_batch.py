"""Batching form: pairs of uneven grid and band advanced together (persistent
sweep kernels over a (pair, tile) work queue, PCG iterations replayed from a
CUDA graph, autotuned tile length).  Each pair's arithmetic equals a single
plan's, so gradients, Hessian-vector products and whole registrations must be
bit-identical to per-pair calls: on six small pairs, and on the 64-pair
workload (grids 64^3 to 160x192x160, bands 16^3 to 32^3) with one pair of every
grid size rerun alone."""

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
