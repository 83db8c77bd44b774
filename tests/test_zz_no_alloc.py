"""glint_env_levels_noalloc, the entry point for callers that cannot allocate
device memory (frame loops that must not stall on cudaMalloc, hosts that own
every allocation), against the allocating path glint_env_create +
glint_env_update on the same maps.  This file is collected last."""
import ctypes

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
    lib = glint.lib
    lib.glint_env_levels_noalloc.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_void_p,
                                             ctypes.c_void_p]
    return glint, render, glint.Context(0), torch, lib


def _allocating_path(gl, env, K, ell):
    glint, render, ctx, torch, lib = gl
    fr = render.Frame(ctx, env, glint.EnvConfig(K=K, ell=ell, out_width=16))
    fr.update_env()
    torch.cuda.synchronize()
    return np.concatenate([fr.env.levels(), fr.env.export(glint.ENV_LOHI)]).astype(np.float64)


def test_noalloc_levels_match_allocating_path(gl):
    glint, render, ctx, torch, lib = gl
    cases = [(synth.env_tiny(0), 4, 1e-4), (synth.env_hdr(seed=3, W=1024, H=512), 8, 1e-4),
             (synth.env_tiny(5), 16, 1e-2)]
    stream = torch.cuda.current_stream().cuda_stream
    for env, K, ell in cases:  # consecutive calls share the library's fixed scratch array
        want = _allocating_path(gl, env, K, ell)
        tex = render.env_tensor(env)
        out = torch.full((K + 2,), -1.0, device="cuda")
        st = lib.glint_env_levels_noalloc(0, tex.data_ptr(), env.width, env.height, render.env_format(env),
                                          env.scale_log2, K, ell, out.data_ptr(), stream)
        assert st == 0, lib.glint_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        assert np.allclose(got, want, rtol=3e-6, atol=0), (got, want)


def test_noalloc_rejects_oversized_and_bad_arguments(gl):
    glint, render, ctx, torch, lib = gl
    out = torch.zeros(10, device="cuda")
    tex = torch.zeros(16, 4, device="cuda")
    assert lib.glint_env_levels_noalloc(0, tex.data_ptr(), 2 * 16384, 16384, 0, 0, 8, 1e-4, out.data_ptr(),
                                        None) == 1
    assert b"maximum" in lib.glint_last_error()
    assert lib.glint_env_levels_noalloc(0, tex.data_ptr(), 8, 4, 0, 0, 3, 1e-4, out.data_ptr(), None) == 1
    assert lib.glint_env_levels_noalloc(0, None, 8, 4, 0, 0, 4, 1e-4, out.data_ptr(), None) == 1
