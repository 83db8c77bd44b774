"""The serving loop on the GPU: each frame's result is the same alone and in
a mix of frames of other resolutions, maps, seeds and paths, and the same as
glint_shade's (bit for bit); frames shaded in place equal uploaded ones;
admission by memory (frames wait for the budget, peak use stays within it);
continuous batching (a small frame submitted after a large one finishes
first)."""
import numpy as np
import pytest

from paper_2507_02674_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_02674_gb300 import build as B
    B.build()
    from paper_2507_02674_gb300 import glint, render
    ctx = glint.Context(0, 64, 128)
    cfg = glint.EnvConfig(K=8, out_width=128)
    frames = [render.Frame(ctx, synth.env_hdr(seed=s, W=256, H=128), cfg) for s in (6, 7)]
    for f in frames:
        f.update_env()
    net = glint.Mlp(ctx, 8, 1024, seed=3)
    net.set_params(synth.mlp_params(seed=4, K=8))
    return glint, render, ctx, torch, frames, net


class Req:
    def __init__(self, torch, render, n, width, seed, pinned=True):
        gb = synth.gbuffer_random(n, seed=seed, width=width)
        self.gb = gb
        self.w, self.h = gb.width, gb.height
        self.planes = render.gbuffer_tensors(gb, device="cpu", pinned=pinned)
        self.tan = torch.from_numpy(gb.tangents())
        self.out = torch.zeros(self.w * self.h, 4)
        if pinned:
            self.tan, self.out = self.tan.pin_memory(), self.out.pin_memory()


def _drain(server, torch, limit=100000):
    done = []
    for _ in range(limit):
        server.tick()
        done += server.poll()
        st = server.stats()
        if st["queued"] == 0 and st["active"] == 0:
            break
    torch.cuda.synchronize()
    return done


def test_alone_equals_mix_equals_glint_shade(gl):
    glint, render, ctx, torch, frames, net = gl
    reqs = [Req(torch, render, 640 * 360, 640, 11), Req(torch, render, 300 * 200, 300, 12),
            Req(torch, render, 1000 * 97 + 13, 1000, 13), Req(torch, render, 50000, 500, 14)]
    plan = [(0, 5, glint.EVAL_E1), (1, 6, glint.EVAL_E1), (0, 7, glint.EVAL_MLP), (1, 8, glint.EVAL_MLP)]

    def server():
        s = glint.Server(ctx, 8, 1 << 30, tick_pixels=100000, tile_pixels=4096)
        s.add_env(frames[0].env, net)
        s.add_env(frames[1].env, net)
        return s

    alone = []
    for r, (e, seed, ev) in zip(reqs, plan):
        s = server()
        s.submit(e, r.planes, r.w, r.h, r.out, seed, ev, r.tan)
        _drain(s, torch)
        alone.append(r.out.clone())
        r.out.zero_()
    s = server()
    for r, (e, seed, ev) in zip(reqs, plan):
        s.submit(e, r.planes, r.w, r.h, r.out, seed, ev, r.tan)
    done = _drain(s, torch)
    assert len(done) == len(reqs)
    st = s.stats()
    assert st["ticks"] > 1 and st["launches"] >= st["ticks"]
    for r, a, (e, seed, ev) in zip(reqs, alone, plan):
        assert torch.equal(r.out, a)  # bit for bit, alone and in the mix
        # and as glint_shade computes the frame on its own
        planes = [p.cuda() for p in r.planes]
        ref = frames[e].shade(planes, r.w, r.h, seed=seed, evaluator=ev, tangent=r.tan.cuda(),
                              mlp=net if ev == glint.EVAL_MLP else None).cpu()
        assert torch.equal(r.out, ref)  # the serving kernels compute each pixel as glint_shade's do


def test_in_place_equals_uploaded(gl):
    """Frames in page-locked memory are shaded in place (no device memory at
    all, on either path); with the server uploading them, or from pageable
    memory (always uploaded), every frame comes out bit for bit the same."""
    glint, render, ctx, torch, frames, net = gl
    shapes = [(640 * 360, 640, 51), (300 * 200 + 7, 300, 52), (50000, 500, 53)]
    plan = [(0, 5, glint.EVAL_E1), (1, 6, glint.EVAL_MLP), (1, 7, glint.EVAL_E1)]
    outs = {}
    for mode in ("in_place", "upload", "pageable"):
        reqs = [Req(torch, render, n, w, sd, pinned=(mode != "pageable")) for n, w, sd in shapes]
        s = glint.Server(ctx, 8, 1 << 30, tick_pixels=100000, tile_pixels=4096, upload=(mode == "upload"))
        s.add_env(frames[0].env, net)
        s.add_env(frames[1].env, net)
        for r, (e, seed, ev) in zip(reqs, plan):
            s.submit(e, r.planes, r.w, r.h, r.out, seed, ev, r.tan)
        assert len(_drain(s, torch)) == len(reqs)
        st = s.stats()
        npix = [r.w * r.h for r in reqs]
        planes = sum(5 * -(-n * 16 // 256) * 256 for n in npix) + -(-npix[1] * 16 // 256) * 256  # + tangent
        assert st["peak_bytes"] == (0 if mode == "in_place" else planes)
        assert st["used_bytes"] == 0
        outs[mode] = [r.out.clone() for r in reqs]
        assert all(bool(o.abs().sum() > 0) for o in outs[mode])
        s.close()
    for a, b, c in zip(outs["in_place"], outs["upload"], outs["pageable"]):
        assert torch.equal(a, b) and torch.equal(a, c)


def test_admission_by_memory(gl):
    glint, render, ctx, torch, frames, net = gl
    r = [Req(torch, render, 640 * 360, 640, 20 + i) for i in range(5)]
    per_frame = 5 * (640 * 360 * 16)  # 4 planes + output (each 256-byte aligned: exact here)
    s = glint.Server(ctx, 8, 2 * per_frame + 4096, tick_pixels=1 << 22, upload=True)
    e = s.add_env(frames[0].env)
    for i, q in enumerate(r):
        s.submit(e, q.planes, q.w, q.h, q.out, i)
    s.tick()
    st = s.stats()
    assert st["active"] == 2 and st["queued"] == 3
    done = _drain(s, torch)
    assert sorted(d[0] for d in done) == [1, 2, 3, 4, 5]
    st = s.stats()
    assert st["peak_bytes"] <= 2 * per_frame + 4096 and st["used_bytes"] == 0
    big = Req(torch, render, 1200 * 600, 1200, 30)
    with pytest.raises(glint.GlintError):  # can never fit
        s.submit(e, big.planes, big.w, big.h, big.out, 0)


def test_continuous_batching_small_frame_overtakes(gl):
    glint, render, ctx, torch, frames, net = gl
    big = Req(torch, render, 2000 * 1000, 2000, 40)
    small = Req(torch, render, 200 * 100, 200, 41)
    s = glint.Server(ctx, 8, 1 << 30, tick_pixels=200000, tile_pixels=16384)
    e = s.add_env(frames[0].env)
    i_big = s.submit(e, big.planes, big.w, big.h, big.out, 1)
    s.tick()
    s.tick()
    i_small = s.submit(e, small.planes, small.w, small.h, small.out, 2)
    done = _drain(s, torch)
    order = [d[0] for d in done]
    assert order.index(i_small) < order.index(i_big)
    t = {d[0]: d for d in done}
    assert t[i_small][2] < t[i_big][3]  # admitted while the big frame was in flight


def test_map_update_between_frames(gl):
    """A map updated while frames are queued: frames submitted before the
    update are shaded with the old map, frames after it with the new one, each
    as glint_shade computes it with that map."""
    glint, render, ctx, torch, frames, net = gl
    cfg = glint.EnvConfig(K=8, out_width=128)
    env_a, env_b = synth.env_hdr(seed=21, W=256, H=128), synth.env_hdr(seed=22, W=256, H=128)
    ref_a, ref_b, served = (render.Frame(ctx, e, cfg) for e in (env_a, env_b, env_a))
    for f in (ref_a, ref_b, served):
        f.update_env()
    reqs = [Req(torch, render, 300 * 200, 300, 50 + i) for i in range(3)]
    s = glint.Server(ctx, 8, 1 << 30, tick_pixels=20000, tile_pixels=4096)
    e = s.add_env(served.env)
    s.submit(e, reqs[0].planes, reqs[0].w, reqs[0].h, reqs[0].out, 1)
    s.tick()
    s.update_env(e, ref_b.texels)
    s.submit(e, reqs[1].planes, reqs[1].w, reqs[1].h, reqs[1].out, 2)
    s.submit(e, reqs[2].planes, reqs[2].w, reqs[2].h, reqs[2].out, 3)
    done = _drain(s, torch)
    assert len(done) == 3
    for r, ref, seed in ((reqs[0], ref_a, 1), (reqs[1], ref_b, 2), (reqs[2], ref_b, 3)):
        want = ref.shade([p.cuda() for p in r.planes], r.w, r.h, seed=seed).cpu()
        assert torch.equal(r.out, want)
