"""ldg_jvp_noalloc: J.v whose scratch is a static device array, for callers that
cannot allocate device memory at the point of the call (an application whose own
pool or caching allocator holds all device memory, or a host loop that cannot wait
on an allocation). Checked through the C-ABI against ldg_jvp, on two calls in a
row, with two contexts sharing the array, and inside a global-mode stream
capture replayed as a CUDA graph. This file is collected last so that
a failure here cannot hide an earlier one."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2205_07824_b300 import synth
from gpu_util import SHEAR2, SHEAR3, assert_parity, cuda, host, pair

pytestmark = pytest.mark.gpu


def _call(g, u, v, out):
    from paper_2205_07824_b300.ldg import lib
    return lib().ldg_jvp_noalloc(g._h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()))


@pytest.mark.parametrize("mesh,p,model,case", [
    (lambda: synth.hex_box((3, 4, 3), affine=SHEAR3), 3, oracle.CONVDIFF, oracle.CASE_EXPSIN),
    (lambda: synth.quad_box((9, 7), affine=SHEAR2), 2, oracle.POISSON, oracle.CASE_SINSIN),
    (lambda: synth.quad_box((6, 5), hi=(10.0, 10.0), periodic=(True, True)), 3, oracle.EULER, oracle.CASE_VORTEX),
])
def test_noalloc_jvp_matches_jvp_twice(mesh, p, model, case):
    import torch
    m = mesh()
    o, g = pair(m, p, model, case, gmres_m=2)
    u = cuda(synth.random_euler_state(m.n_elem, o.npe, 3) if model == oracle.EULER else synth.random_vector(o.ndof, 3))
    v = cuda(synth.random_vector(o.ndof, 4))
    ref = host(g.jvp(u, v))
    for _ in range(2):
        out = torch.full_like(u, float("nan"))
        assert _call(g, u, v, out) == 0
        assert_parity(host(out), ref, what="jvp_noalloc")
    # the same operator with a second direction: the array's old contents do not leak in
    v2 = cuda(synth.random_vector(o.ndof, 5))
    out = torch.empty_like(u)
    assert _call(g, u, v2, out) == 0
    assert_parity(host(out), host(g.jvp(u, v2)), what="jvp_noalloc second direction")


def test_noalloc_two_contexts_share_the_array():
    """Two contexts on one device (different meshes, orders and models) take turns on
    the one static array, A then B then A on one stream; each result equals that
    context's own ldg_jvp."""
    import torch
    ma = synth.hex_box((3, 2, 3), affine=SHEAR3)
    mb = synth.quad_box((5, 4), hi=(2.0, 2.0), periodic=(True, True))
    oa, ga = pair(ma, 2, oracle.CONVDIFF, oracle.CASE_EXPSIN, gmres_m=2)
    ob, gb = pair(mb, 3, oracle.NS, oracle.CASE_ROTATION, gmres_m=2)
    ua, va = cuda(synth.random_vector(oa.ndof, 6)), cuda(synth.random_vector(oa.ndof, 7))
    ub = cuda(synth.random_euler_state(mb.n_elem, ob.npe, 8))
    vb = cuda(synth.random_vector(ob.ndof, 9))
    ref_a, ref_b = host(ga.jvp(ua, va)), host(gb.jvp(ub, vb))
    for g, u, v, ref, what in ((ga, ua, va, ref_a, "A"), (gb, ub, vb, ref_b, "B"), (ga, ua, va, ref_a, "A again")):
        out = torch.full_like(u, float("nan"))
        assert _call(g, u, v, out) == 0
        assert_parity(host(out), ref, what=f"jvp_noalloc context {what}")


def test_noalloc_rejects_operators_beyond_the_static_maximum():
    from paper_2205_07824_b300.ldg import LDG, lib
    import torch
    m = synth.hex_box(32)   # 32768 hexahedra, p = 3: n_dof * dim = 6.3 M doubles > 4 Mi
    g = LDG(m, 3, oracle.CONVDIFF, oracle.CASE_EXPSIN, (0.01, 0.01, 1.0, 0.5, 0.25), gmres_m=1)
    u = torch.zeros(g.n_dof, dtype=torch.float64, device="cuda")
    rc = _call(g, u, u, torch.empty_like(u))
    assert rc == -1
    msg = lib().ldg_last_error(g._h).decode()
    assert "4194304" in msg and str(g.n_dof * 3) in msg


@pytest.mark.parametrize("which", ["convdiff_hex", "ns_quad"])
def test_noalloc_jvp_inside_global_stream_capture(which):
    """The entry point allocates nothing once the device's array address is known:
    after one call outside a capture, a call inside a global-mode stream capture
    (where an allocation anywhere in the process invalidates the capture) records,
    the graph replays, and its J.v equals the context's own ldg_jvp."""
    import torch
    if which == "convdiff_hex":
        o, g = pair(synth.hex_box((3, 4, 3), affine=SHEAR3), 3, oracle.CONVDIFF, oracle.CASE_EXPSIN, gmres_m=2)
        u = cuda(synth.random_vector(o.ndof, 21))
    else:
        m = synth.quad_box((5, 4), hi=(2.0, 2.0), periodic=(True, True))
        o, g = pair(m, 3, oracle.NS, oracle.CASE_ROTATION, gmres_m=2)
        u = cuda(synth.random_euler_state(m.n_elem, o.npe, 22))
    v = cuda(synth.random_vector(o.ndof, 23))
    ref = host(g.jvp(u, v))
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g.set_stream(s)
    out = torch.full_like(u, float("nan"))
    with torch.cuda.stream(s):
        assert _call(g, u, v, out) == 0
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s, capture_error_mode="global"):
        rc = _call(g, u, v, out)
    assert rc == 0
    with torch.cuda.stream(s):
        out.fill_(float("nan"))
        graph.replay()
    s.synchronize()
    assert_parity(host(out), ref, what=f"jvp_noalloc replayed from a global-mode capture ({which})")
