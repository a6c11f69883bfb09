"""Batched persistent launch: many uneven cubes, each with its own camera,
table and image, in one launch (optionally a CUDA graph).  Results must equal
the per-job vr_render outputs and the oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import TOL_F32, compare, cuda_or_skip

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def P(torch):
    import paper_1211_4896_gb300 as P
    return P


def _jobs(torch, P, n=7, store="f16"):
    dev = torch.device("cuda")
    rng = np.random.default_rng(42)
    jobs, cubes = [], []
    for q in range(n):
        dims = tuple(int(x) for x in rng.integers(12, 60, size=3))
        cube = synth.hi_cube(dims, n_blobs=4, n_disks=1, seed=700 + q)
        vol = P.Volume(cube.to(dev), store)
        W, H = int(rng.integers(9, 70)), int(rng.integers(7, 66))
        cam = synth.camera_random_persp(dims, seed=800 + q, width=W, height=H)
        tf_np = synth.tf_random_pwl(seed=900 + q)
        jobs.append(dict(vol=vol, cam=cam, tf=torch.from_numpy(tf_np).to(dev), tf_np=tf_np, vmin=-3.0, vmax=30.0,
                         step=0.5 + 0.1 * (q % 3), ert=0.99 if q % 2 else 2.0,
                         out=torch.full((H, W, 4), -1.0, device=dev),
                         nsamples=torch.full((H, W), -1, dtype=torch.int32, device=dev)))
        cubes.append(cube)
    return jobs, cubes


@pytest.mark.parametrize("use_graph", [False, True])
def test_batched_equals_single_renders(P, torch, use_graph):
    jobs, cubes = _jobs(torch, P)
    P.render_batched(jobs, use_graph=use_graph)
    P.render_batched(jobs, use_graph=use_graph)          # replay: same result
    torch.cuda.synchronize()
    for j, cube in zip(jobs, cubes):
        img, ns = P.render(j["vol"], j["cam"], j["tf"], j["vmin"], j["vmax"], j["step"], j["ert"])
        torch.cuda.synchronize()
        assert torch.equal(j["out"], img)
        assert torch.equal(j["nsamples"], ns)
    # and the oracle, on the rounded cubes the kernel reads
    for j, cube in list(zip(jobs, cubes))[:3]:
        bits = cube.to(torch.float16).view(torch.int16).numpy().view(np.uint16)
        ref = oracle.render(bits, j["cam"], j["tf_np"], j["vmin"], j["vmax"], j["step"], j["ert"], bits="f16")
        compare(j["out"].cpu().numpy(), j["nsamples"].cpu().numpy(), ref, TOL_F32)
    for j in jobs:
        j["vol"].close()


@pytest.mark.parametrize("tile", [(4, 8), (16, 2), (32, 1)])
def test_batched_tile_shapes(P, torch, tile):
    jobs, _ = _jobs(torch, P, n=4, store="f32")
    P.render_batched(jobs, use_graph=False, tile=tile, ctas_per_sm=2)
    torch.cuda.synchronize()
    for j in jobs:
        img, ns = P.render(j["vol"], j["cam"], j["tf"], j["vmin"], j["vmax"], j["step"], j["ert"])
        torch.cuda.synchronize()
        assert torch.equal(j["out"], img)
        j["vol"].close()


def test_autotune_and_validation(P, torch):
    from paper_1211_4896_gb300 import _lib as L
    jobs, _ = _jobs(torch, P, n=3, store="f32")
    cj = P.render_batched(jobs, use_graph=False)
    best = L.vr_autotune_batched(cj, L.vr_batch_opts(1, 0, 0, 0))
    assert best.tile_w * best.tile_h == 32 and best.use_graph == 1
    # mixed storage types in one batch are rejected before any launch
    dev = torch.device("cuda")
    other = P.Volume(torch.zeros((8, 8, 8), device=dev), "f16")
    jobs[1] = dict(jobs[1], vol=other)
    with pytest.raises(P.VRError) as ei:
        P.render_batched(jobs, use_graph=False)
    assert ei.value.status == -2
    with pytest.raises(P.VRError):
        P.render_batched(jobs[:1], tile=(5, 6))
    for j in jobs:
        j["vol"].close()


def test_autotune_cache_round_trip(P, torch, tmp_path):
    """The tuned options are stored under the job list's key and read back
    (no second tuning); rendering with them equals single renders."""
    import json
    jobs, _ = _jobs(torch, P, n=3, store="f16")
    path = str(tmp_path / "tune.json")
    a = P.autotune_batched(jobs, cache_path=path)
    table = json.load(open(path))
    assert list(table) == [P.api.autotune_key(jobs)]
    table[P.api.autotune_key(jobs)]["ctas_per_sm"] = 2          # a hit returns the stored entry as is
    json.dump(table, open(path, "w"))
    b = P.autotune_batched(jobs, cache_path=path)
    assert (b.tile_w, b.tile_h, b.ctas_per_sm) == (a.tile_w, a.tile_h, 2)
    assert a.tile_w * a.tile_h == 32
    P.render_batched(jobs, opts=b)
    torch.cuda.synchronize()
    for j in jobs:
        img, ns = P.render(j["vol"], j["cam"], j["tf"], j["vmin"], j["vmax"], j["step"], j["ert"])
        assert torch.equal(j["out"], img) and torch.equal(j["nsamples"], ns)
        j["vol"].close()


@pytest.mark.parametrize("store", ["f32", "f16"])
@pytest.mark.parametrize("wpt,tile", [(2, (8, 4)), (4, (8, 4)), (2, (16, 2)), (4, (32, 1))])
def test_warps_sharing_a_tile_equal_single_renders(P, torch, store, wpt, tile):
    """Two or four warps of a CTA take one tile together (each its own part,
    handed over at a named barrier of the group): the images equal the single
    renders bit for bit, with the graph replayed."""
    from paper_1211_4896_gb300 import _lib as L
    jobs, _ = _jobs(torch, P, n=5, store=store)
    opts = L.vr_batch_opts(1, tile[0], tile[1], 0, wpt)
    for _ in range(2):
        for j in jobs:
            j["out"].fill_(-1.0)
            j["nsamples"].fill_(-1)
        P.render_batched(jobs, opts=opts)
        torch.cuda.synchronize()
        for j in jobs:
            img, ns = P.render(j["vol"], j["cam"], j["tf"], j["vmin"], j["vmax"], j["step"], j["ert"])
            torch.cuda.synchronize()
            assert torch.equal(j["out"], img) and torch.equal(j["nsamples"], ns)
    with pytest.raises(P.VRError):
        P.render_batched(jobs, opts=L.vr_batch_opts(0, 8, 4, 0, 3))
    for j in jobs:
        j["vol"].close()


@pytest.mark.parametrize("store", ["f32", "f16"])
def test_rebrick_renders_like_the_source(P, torch, store):
    """vr_volume_rebrick builds bricks of another size from a volume's bricks:
    renders from 32^3 and 64^3 bricks (and back to 16^3) equal the source's
    and those of a volume created with that size from the dense cube."""
    jobs, cubes = _jobs(torch, P, n=3, store=store)
    for j, cube in zip(jobs, cubes):
        ref, ref_ns = P.render(j["vol"], j["cam"], j["tf"], j["vmin"], j["vmax"], j["step"], j["ert"])
        for b in (32, 64):
            rb = j["vol"].rebrick(b)
            direct = P.Volume(cube.cuda(), store, brick=b)
            back = rb.rebrick(16)
            assert rb.info["brick"] == b and rb.info["dims"] == j["vol"].info["dims"]
            for v in (rb, direct, back):
                img, ns = P.render(v, j["cam"], j["tf"], j["vmin"], j["vmax"], j["step"], j["ert"])
                torch.cuda.synchronize()
                assert torch.equal(img, ref) and torch.equal(ns, ref_ns)
            for v in (rb, direct, back):
                v.close()
        with pytest.raises(P.VRError):
            j["vol"].rebrick(8)
        j["vol"].close()


def test_autotune_over_brick_sizes(P, torch, tmp_path):
    """The autotuner over brick sizes returns options, a brick size and the
    job list on volumes of that size; rendering with them equals the single
    renders; the cache entries record brick size and warps per tile."""
    import json
    jobs, _ = _jobs(torch, P, n=4, store="f16")
    path = str(tmp_path / "tune.json")
    opts, brick, tuned = P.autotune_batched_bricks(jobs, brick_sizes=(16, 32), cache_path=path)
    assert brick in (16, 32) and opts.warps_per_tile in (1, 2, 4) and opts.tile_w * opts.tile_h == 32
    assert all(int(j["vol"].info["brick"]) == brick for j in tuned)
    table = json.load(open(path))
    assert len(table) == 2 and {e["brick"] for e in table.values()} == {16, 32}
    assert all("warps_per_tile" in e for e in table.values())
    P.render_batched(tuned, opts=opts)
    torch.cuda.synchronize()
    for j in tuned:
        img, ns = P.render(j["vol"], j["cam"], j["tf"], j["vmin"], j["vmax"], j["step"], j["ert"])
        torch.cuda.synchronize()
        assert torch.equal(j["out"], img) and torch.equal(j["nsamples"], ns)
    for j in jobs:
        for v in j["vol"].__dict__.get("_rebricked", {}).values():
            v.close()
        j["vol"].close()
