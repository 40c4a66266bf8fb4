"""gsrf_render_static: the render for callers that cannot allocate device memory.

Its workspace is a fixed array compiled into the library instead of a buffer the
caller allocates.  These checks call it through the C ABI twice in a row, on two
different problems, and hold each result to the output of the ordinary entry point
(gsrf_render with a caller-allocated workspace) at the tolerance the parity tests use;
they also check that a problem too large for the array is refused before any launch.
This file is collected last so that a run stopping at the first failure has already
run every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2502_01826_gb300 import _lib as L
from paper_2502_01826_gb300 import synthetic
from paper_2502_01826_gb300.render import Renderer, gaussians_struct, make_grid, to_device

from gpu_util import TOL_L2

pytestmark = pytest.mark.gpu


def _problem(K, spec, seed):
    scene = synthetic.tiny_scene(K, seed, box=(8.0, 6.0, 3.0))
    rng = np.random.default_rng(seed)
    rx = (rng.uniform(0, 1, (1, 3)) * [8.0, 6.0, 3.0]).astype(np.float32)
    tx = (rng.uniform(0, 1, 3) * [8.0, 6.0, 3.0]).astype(np.float32)
    return scene, rx, tx, make_grid(**spec)


def _render_both(scene, rx, tx, grid, f0=2.4e9):
    lib = L.load(build_if_missing=True)
    K = scene["means"].shape[0]
    p = to_device(scene)
    rxd = torch.tensor(rx, device="cuda")
    txd = torch.tensor(tx, device="cuda")
    R = Renderer(K, 1, grid, f0)
    R.ensure_capacity(p, rxd, txd)
    ref = R.forward(p, rxd, txd)  # gsrf_render, caller-allocated workspace
    out = torch.full(R.out_shape(), float("nan"), dtype=torch.float32, device="cuda")
    gs = gaussians_struct(p)
    st = L.gsrf_run_status()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = lib.gsrf_render_static(C.byref(R.plan), C.byref(gs), C.c_void_p(rxd.data_ptr()),
                                  C.c_void_p(txd.data_ptr()), C.c_void_p(out.data_ptr()), C.byref(st), stream)
    assert code == L.GSRF_OK, L.STATUS_NAMES.get(code, code)
    assert st.code == L.GSRF_OK and st.required_pairs > 0
    torch.cuda.synchronize()
    return out.cpu().numpy(), ref.cpu().numpy()


def test_static_scratch_render_matches_allocated_workspace_twice():
    # two calls in a row on different problems: the second runs over the first's leftovers
    cases = [(2048, dict(n_az=36, n_el=9), 11), (6000, dict(n_az=72, n_el=18), 12)]
    for K, spec, seed in cases:
        scene, rx, tx, grid = _problem(K, spec, seed)
        got, ref = _render_both(scene, rx, tx, grid)
        assert np.all(np.isfinite(got))
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= TOL_L2, err
        assert np.count_nonzero(ref) > 0


def test_static_scratch_refuses_problems_beyond_its_size():
    lib = L.load(build_if_missing=True)
    grid = make_grid(360, 90)
    plan = L.gsrf_plan(2_000_000, 4, 1, 2.4e9, 0.0, grid, 50_000_000)
    need = C.c_size_t()
    assert lib.gsrf_workspace_size(C.byref(plan), C.byref(need)) == L.GSRF_OK
    assert need.value > L.GSRF_STATIC_SCRATCH_BYTES
    g = L.gsrf_gaussians(2_000_000, 256, 256, 256, 256, 256, None)
    out = C.c_void_p(256)
    code = lib.gsrf_render_static(C.byref(plan), C.byref(g), C.c_void_p(256), C.c_void_p(256), out, None, None)
    assert code == L.GSRF_ERR_TOO_LARGE
