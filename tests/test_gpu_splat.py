"""GPU Gaussian-splatting render against the oracle's float64 restatement of the
3DGS forward equations.  Float32 may take a discrete decision of the forward the
other way where float64 puts it within float32 reach of its threshold (the 1/255
alpha floor, the 0.99 cap, the 1e-4 transmittance stop, the 3-sigma radius and
tile square, the depth order of near-equal depths); the oracle flags those pixels
(orc_gs_render_flags) and they are counted.  Every other pixel, colour and
transmittance, must agree within PIXEL_TOL, the mean error within MEAN_TOL, and
closed-form scenes within 1e-5."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_00444_gb300 import MeshBVH, gs_render
from parity import dev, host
from workloads.meshes import icosphere, torus, TorusSkinning
from workloads.sampling import osada_barycentrics

pytestmark = pytest.mark.gpu


def look_at(eye, target, up=(0, 0, 1)):
    eye, target, up = (np.asarray(x, np.float64) for x in (eye, target, up))
    z = target - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, up)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    return R, -R @ eye


# Both sides render the same float32 inputs; the kernel's float32 arithmetic moves a
# projected centre by a few ulp (~1e-5 pixel at ~100 pixels from the principal point), an
# exponent p by ~1e-5 and an alpha by ~1e-5 of itself, and a pixel's colour is a sum of
# alpha-weighted colours of total weight at most 1: unflagged pixels agree to a few 1e-6
# (measured: at most 1.8e-6 over these scenes), so PIXEL_TOL = 1e-5.  The oracle flags a
# per-pixel threshold within MARGIN (relative) of its value, 4x the alpha error bound for
# images up to 128 pixels (scaled with the image size beyond).  Dense face-bound scenes flag
# up to ~10 % of their pixels (mostly near-equal depths of overlapping Gaussians, where the
# order or the transmittance stop may fall the other way).
PIXEL_TOL = 1e-5
MEAN_TOL = 2e-5
MARGIN = 2e-4
FLAGGED_MAX = 0.12


def compare(args, cam, W, H, bg=(0.05, 0.1, 0.2), strict=None):
    mu, quat, scale, opac, col = args
    R, t, f = cam
    img, T = gs_render(*(dev(np.asarray(a, np.float32)) for a in args), R, t, f, f, W / 2, H / 2, W, H,
                       background=bg)
    # the oracle renders the float32 inputs the kernel was given (camera included), in float64
    f32 = lambda a: np.asarray(np.asarray(a, np.float32), np.float64)   # noqa: E731
    rimg, rT, frag = oracle.gs_render(*(f32(a) for a in args), f32(R), f32(t), float(np.float32(f)),
                                      float(np.float32(f)), W / 2, H / 2, W, H, 0.01, f32(bg), flags=True,
                                      margin=MARGIN * max(1.0, max(W, H) / 128))
    err = np.abs(host(img) - rimg).max(2)
    terr = np.abs(host(T) - rT)
    if strict is not None:
        assert err.max() <= strict and terr.max() <= strict
        return
    ok = ~frag
    worst = np.unravel_index(np.argmax(np.where(ok, terr + err, -1.0)), err.shape)
    print(f"flagged {frag.mean():.4%} of {frag.size} pixels; unflagged max colour error "
          f"{err[ok].max():.3g}, transmittance {terr[ok].max():.3g}; mean {err.mean():.3g}; worst unflagged "
          f"pixel {tuple(int(x) for x in worst)}: T {float(host(T)[worst]):.6g} vs {float(rT[worst]):.6g}")
    assert frag.mean() <= FLAGGED_MAX
    assert err[ok].max() <= PIXEL_TOL and terr[ok].max() <= PIXEL_TOL
    assert err.mean() <= MEAN_TOL


def random_gaussians(n, seed):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-1, 1, (n, 3)) * [1.0, 0.7, 0.5]
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    scale = rng.uniform(0.01, 0.12, (n, 3))
    return mu, q, scale, rng.uniform(0.1, 0.95, n), rng.uniform(0, 1, (n, 3))


def test_random_gaussians_ragged_image():
    R, t = look_at([0.3, -3.0, 0.8], [0, 0, 0])
    compare(random_gaussians(300, 1), (R, t, 90.0), 100, 70)


def test_one_isotropic_gaussian_closed_form():
    I3, Z3 = np.eye(3), np.zeros(3)
    args = ([[0, 0, 2.0]], [[1, 0, 0, 0]], [[0.2, 0.2, 0.2]], [0.8], [[0.9, 0.5, 0.1]])
    compare(tuple(np.array(a, float) for a in args), (I3, Z3, 40.0), 32, 32, bg=(0.1, 0.2, 0.3), strict=1e-5)


def test_face_bound_gaussians_of_a_mesh():
    """The rebind kernel's output rendered: the path from mesh to image."""
    V, F = icosphere(3)
    rng = np.random.default_rng(2)
    gface = np.repeat(np.arange(F.shape[0], dtype=np.int32), 2)
    gbary = osada_barycentrics(rng, gface.shape[0]).astype(np.float32)
    bvh = MeshBVH.from_mesh(dev(V), dev(F))
    mu, quat, scale = (host(x).astype(np.float64) for x in bvh.bind_gaussians(dev(gface), dev(gbary)))
    opac = rng.uniform(0.5, 0.9, gface.shape[0])
    col = rng.uniform(0, 1, (gface.shape[0], 3))
    R, t = look_at([2.2, -1.5, 1.0], [0, 0, 0])
    compare((mu, quat, scale * 3.0, opac, col), (R, t, 80.0), 96, 80)


def test_empty_and_culled():
    R, t = look_at([0, -3, 0], [0, 0, 0])
    img, T = gs_render(*(dev(np.zeros((0, k), np.float32)) for k in (3, 4, 3)), dev(np.zeros(0, np.float32)),
                       dev(np.zeros((0, 3), np.float32)), R, t, 50, 50, 20, 20, 40, 40, background=(0.5, 0.25, 1.0))
    assert torch.allclose(img, torch.tensor([0.5, 0.25, 1.0], device="cuda").expand_as(img))
    assert (host(T) == 1).all()


def test_torus_gaussians_subset_full_pipeline():
    """Gaussians of the skinned 200k-face torus (every 15th of 600k), 128 x 96 view."""
    V0, F = torus(400, 250)
    V = TorusSkinning(V0, seed=3000).frame(20)
    rng = np.random.default_rng(3)
    gface = np.repeat(np.arange(F.shape[0], dtype=np.int32), 3)[::15].copy()
    gbary = osada_barycentrics(rng, gface.shape[0]).astype(np.float32)
    bvh = MeshBVH.from_mesh(dev(V), dev(F))
    mu, quat, scale = (host(x).astype(np.float64) for x in bvh.bind_gaussians(dev(gface), dev(gbary)))
    opac = rng.uniform(0.3, 0.9, gface.shape[0])
    col = rng.uniform(0, 1, (gface.shape[0], 3))
    R, t = look_at([0.5, -2.8, 1.6], [0, 0, 0])
    compare((mu, quat, scale * 4.0, opac, col), (R, t, 110.0), 128, 96)


def test_fixed_capacity_render_is_the_render_and_replays_in_a_graph():
    """mesh_gs_render_capacity (no host read of the instance count): with room for every
    instance it draws mesh_gs_render's image bit for bit and reports the count; captured
    in a CUDA graph it follows new Gaussian positions on replay; past its capacity it
    flags the overflow."""
    from paper_2606_00444_gb300 import gs_render_capacity
    W, H, f = 160, 96, 120.0
    R, t = look_at([0.3, -3.0, 0.8], [0, 0, 0])
    mu, q, sc, op, col = (dev(np.asarray(a, np.float32)) for a in random_gaussians(500, 7))
    img, T = gs_render(mu, q, sc, op, col, R, t, f, f, W / 2, H / 2, W, H)
    counts = torch.zeros(2, dtype=torch.int32, device="cuda")
    cimg, cT, _ = gs_render_capacity(mu, q, sc, op, col, R, t, f, f, W / 2, H / 2, W, H, 200000, counts=counts)
    torch.cuda.synchronize()
    n_inst = int(counts[1].item())
    assert counts[0].item() == 0 and n_inst > 500
    assert torch.equal(cimg, img) and torch.equal(cT, T)
    # exactly enough room, and a graph replay after the Gaussians moved
    from paper_2606_00444_gb300 import Workspace
    ws = Workspace(torch.device("cuda"))
    out = (torch.empty_like(img), torch.empty_like(T))
    cap = n_inst + 64
    gs_render_capacity(mu, q, sc, op, col, R, t, f, f, W / 2, H / 2, W, H, cap, ws=ws, out=out, counts=counts)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        gs_render_capacity(mu, q, sc, op, col, R, t, f, f, W / 2, H / 2, W, H, cap, ws=ws, out=out,
                           counts=counts)
    mu2 = mu + torch.tensor([0.05, 0.0, -0.03], device="cuda")
    mu.copy_(mu2)
    g.replay()
    torch.cuda.synchronize()
    img2, T2 = gs_render(mu, q, sc, op, col, R, t, f, f, W / 2, H / 2, W, H)
    if counts[0].item() == 0:
        assert torch.equal(out[0], img2) and torch.equal(out[1], T2)
    # too little room: the overflow is flagged and the count still reported
    small = max(1, n_inst // 3)
    gs_render_capacity(mu, q, sc, op, col, R, t, f, f, W / 2, H / 2, W, H, small, counts=counts)
    torch.cuda.synchronize()
    assert counts[0].item() == 1 and counts[1].item() > small
