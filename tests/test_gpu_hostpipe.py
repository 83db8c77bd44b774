"""Shading a frame held in host memory (glint_shade_host) gives glint_shade's
frame bit for bit, both ways: in place (page-locked buffers read and written
by the kernels over the host link, one launch) and staged (bands of whole rows
uploaded, shaded and downloaded on three streams) -- for the default bands and
for bands with a ragged last one, 2, 3 and 8 staging slots, pinned and
pageable host buffers (pageable ones, or a mix, are always staged), the E1, E2
and surrogate evaluators, and calls in a row on one pipe (with and without
the inputs-ready flag, which lets staged uploads start before the stream's
earlier work); sizes the pipe cannot hold are rejected."""
import pytest

from paper_2507_02674_gb300 import synth

pytestmark = pytest.mark.gpu

W, H = 640, 360


@pytest.fixture(scope="module")
def gl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_02674_gb300 import build as B
    B.build()
    from paper_2507_02674_gb300 import glint, render
    ctx = glint.Context(0, 64, 128)
    fr = render.Frame(ctx, synth.env_hdr(seed=6, W=256, H=128), glint.EnvConfig(K=8, out_width=128))
    fr.update_env()
    gb = synth.gbuffer_random(W * H, seed=41, width=W)
    assert (gb.width, gb.height) == (W, H)
    net = glint.Mlp(ctx, 8, 1024, seed=3)
    net.set_params(synth.mlp_params(seed=4, K=8))
    host = render.gbuffer_tensors(gb, device="cpu", pinned=True)
    tan = torch.from_numpy(gb.tangents()).pin_memory()
    return glint, render, torch, ctx, fr, gb, net, host, tan


def _direct(torch, fr, host, tan, seed, evaluator, net, e2_samples=4):
    planes = [p.cuda() for p in host]
    out = fr.shade(planes, W, H, seed=seed, evaluator=evaluator, tangent=tan.cuda(), mlp=net, e2_samples=e2_samples)
    torch.cuda.synchronize()
    return out.cpu()


@pytest.mark.parametrize("rows_per_band,slots,pinned", [(0, 2, True), (7, 3, True), (64, 2, False), (45, 8, True)])
def test_e1_bands_equal_glint_shade(gl, rows_per_band, slots, pinned):
    glint, render, torch, ctx, fr, gb, net, host, tan = gl
    planes = host if pinned else [p.clone() for p in host]
    pipe = glint.HostPipe(ctx, band_pixels=W * 64, slots=slots)
    out = torch.full((W * H, 4), -1.0)
    if pinned:
        out = out.pin_memory()
    pipe.shade(fr.env, planes, W, H, out, seed=5, rows_per_band=rows_per_band, staged=True)
    torch.cuda.synchronize()
    ref = _direct(torch, fr, host, tan, 5, glint.EVAL_E1, None)
    assert torch.equal(out, ref)
    assert not pipe.last_in_place()
    rpb = rows_per_band or min(64, (H + 7) // 8)
    assert pipe.last_launches() == (H + rpb - 1) // rpb  # one shading launch per band
    pipe.close()


def test_in_place_for_pinned_buffers(gl):
    glint, render, torch, ctx, fr, gb, net, host, tan = gl
    pipe = glint.HostPipe(ctx, band_pixels=W * 8, slots=2)
    out = torch.full((W * H, 4), -1.0).pin_memory()
    for seed in (21, 22):  # two calls in a row on the same buffers
        pipe.shade(fr.env, host, W, H, out, seed=seed)
        torch.cuda.synchronize()
        assert pipe.last_in_place() and pipe.last_launches() == 1
        assert torch.equal(out, _direct(torch, fr, host, tan, seed, glint.EVAL_E1, None))
    # one pageable buffer (here the output) sends the frame through the bands
    pageable = torch.zeros(W * H, 4)
    pipe.shade(fr.env, host, W, H, pageable, seed=21)
    torch.cuda.synchronize()
    assert not pipe.last_in_place()
    assert torch.equal(pageable, _direct(torch, fr, host, tan, 21, glint.EVAL_E1, None))


@pytest.mark.parametrize("evaluator,staged", [("e2", False), ("e2", True), ("mlp", False), ("mlp", True)])
def test_other_evaluators_equal_glint_shade(gl, evaluator, staged):
    glint, render, torch, ctx, fr, gb, net, host, tan = gl
    ev = glint.EVAL_E2 if evaluator == "e2" else glint.EVAL_MLP
    pipe = glint.HostPipe(ctx, band_pixels=W * 50, slots=2)
    out = torch.zeros(W * H, 4).pin_memory()
    p_scratch = torch.empty(W * H, 8, device="cuda") if ev == glint.EVAL_MLP else None
    pipe.shade(fr.env, host, W, H, out, seed=9, tangent=tan, evaluator=ev, e2_samples=4,
               mlp=net if ev == glint.EVAL_MLP else None, p_scratch=p_scratch, rows_per_band=50, staged=staged)
    torch.cuda.synchronize()
    assert pipe.last_in_place() == (not staged)
    ref = _direct(torch, fr, host, tan, 9, ev, net if ev == glint.EVAL_MLP else None)
    assert torch.equal(out, ref)


def test_calls_in_a_row_reuse_the_staging(gl):
    glint, render, torch, ctx, fr, gb, net, host, tan = gl
    pipe = glint.HostPipe(ctx, band_pixels=W * 16, slots=2)
    outs = [torch.zeros(W * H, 4).pin_memory() for _ in range(3)]
    for i, o in enumerate(outs):  # enqueued back to back, no synchronisation between calls
        pipe.shade(fr.env, host, W, H, o, seed=100 + i, rows_per_band=16, inputs_ready=(i % 2 == 1), staged=True)
    torch.cuda.synchronize()
    for i, o in enumerate(outs):
        assert torch.equal(o, _direct(torch, fr, host, tan, 100 + i, glint.EVAL_E1, None))


def test_sizes_the_pipe_cannot_hold_are_rejected(gl):
    glint, render, torch, ctx, fr, gb, net, host, tan = gl
    out = torch.zeros(W * H, 4).pin_memory()
    small = glint.HostPipe(ctx, band_pixels=W - 1, slots=2)
    with pytest.raises(glint.GlintError):  # a row does not fit a band
        small.shade(fr.env, host, W, H, out, staged=True)
    pipe = glint.HostPipe(ctx, band_pixels=W * 10, slots=2)
    with pytest.raises(glint.GlintError):  # 11 rows per band exceed the staging
        pipe.shade(fr.env, host, W, H, out, rows_per_band=11, staged=True)
    with pytest.raises(glint.GlintError):
        glint.HostPipe(ctx, band_pixels=1024, slots=17)
    pipe.shade(fr.env, host, W, 0, out)  # an empty frame is a no-op
    assert pipe.last_launches() == 0


def test_device_buffers_are_staged_and_equal(gl):
    """Buffers that are not host memory at all (device tensors) go through the
    staged path, whose copies take their direction from the addresses."""
    glint, render, torch, ctx, fr, gb, net, host, tan = gl
    planes = [p.cuda() for p in host]
    out = torch.zeros(W * H, 4, device="cuda")
    pipe = glint.HostPipe(ctx, band_pixels=W * 64, slots=2)
    pipe.shade(fr.env, planes, W, H, out, seed=33)
    torch.cuda.synchronize()
    assert not pipe.last_in_place()
    assert torch.equal(out.cpu(), _direct(torch, fr, host, tan, 33, glint.EVAL_E1, None))
