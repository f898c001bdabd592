"""The allocation-free entry point rs_gram_noalloc against the oracle and the context path.

Callers that cannot allocate device memory (a host application that has reserved all of it,
a latency-critical path where an allocation may synchronise the device, a plug-in limited
to the memory it is handed) use rs_gram_noalloc, whose scratch is a fixed array inside the
library.  This file is collected last so that a stop at the first failure has already run
every other test; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import rs_oracle as O  # noqa: E402
from workloads import load_config, make_particles  # noqa: E402

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12   # FP64 Gram matrices (the FP32 bulk path forms G in double-float arithmetic, ~1e-14)


def _gram_noalloc(lib, ccfg, xyz, Z, n):
    G = torch.empty((3, n, n), dtype=torch.float64, device="cuda")
    st = lib.rs_gram_noalloc(C.byref(ccfg), int(Z.numel()), C.c_void_p(xyz.data_ptr()),
                             C.c_void_p(Z.data_ptr()), C.c_void_p(G.data_ptr()),
                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, G


@pytest.mark.parametrize("name", ["c1_box64_n129", "c2_protein1000_n513"])
def test_noalloc_gram_matches_context_path_twice(name):
    from paper_1606_09218_gb300 import RSContext, _lib, config_from_workload
    lib = _lib.load()
    cfg = load_config(name)
    p = make_particles(cfg)
    n = int(cfg["n"])
    xyz = torch.tensor(p.xyz, device="cuda")
    Z = torch.tensor(p.Z, device="cuda")
    ccfg = config_from_workload(cfg, max_particles=len(p.Z))
    ctx = RSContext(ccfg)
    ctx.solve(xyz, Z, energy=False, want_potential=False)
    G_ref = ctx.debug_buffer("G", torch.float64)[: 3 * n * n].view(3, n, n).clone()
    ctx.close()
    for call in range(2):                       # two calls in a row share the scratch array
        st, G = _gram_noalloc(lib, ccfg, xyz, Z, n)
        assert st == _lib.RS_OK, lib.rs_last_error(None)
        torch.cuda.synchronize()
        err = float((G - G_ref).norm() / G_ref.norm())
        assert err < REL_TOL, (call, err)


def test_noalloc_gram_matches_oracle_side_matrices():
    """G_l = U^(l) U^(l)^T with the oracle's side matrices (Sec. 3.2, Eq. (3.5)), per mode."""
    from paper_1606_09218_gb300 import _lib, config_from_workload
    lib = _lib.load()
    cfg = load_config("c1_box64_n129")
    p = make_particles(cfg)
    n = int(cfg["n"])
    pr = O.Problem(cfg, p.xyz, p.Z)
    Us, _ = O.side_matrices(pr.j, pr.z, pr.pk, pr.klong, n)
    ccfg = config_from_workload(cfg, max_particles=len(p.Z))
    st, G = _gram_noalloc(lib, ccfg, torch.tensor(p.xyz, device="cuda"), torch.tensor(p.Z, device="cuda"), n)
    assert st == _lib.RS_OK, lib.rs_last_error(None)
    G = G.cpu().numpy()
    for l in range(3):
        ref = Us[l] @ Us[l].T
        assert np.linalg.norm(G[l] - ref) <= REL_TOL * np.linalg.norm(ref), l


def test_noalloc_rejects_a_centre_outside_the_box_like_the_context_path():
    """A centre just outside [-b, b]^3 (and a non-finite charge) is an error, as in rs_solve."""
    from paper_1606_09218_gb300 import RSContext, RSError, _lib, config_from_workload
    lib = _lib.load()
    cfg = dict(load_config("c1_box64_n129"))
    b, n = float(cfg["b"]), int(cfg["n"])
    ccfg = config_from_workload(cfg, max_particles=3)
    xyz = torch.tensor([[0.0, 0.0, 0.0], [1.0, -2.0, 3.0], [b * (1 + 1e-9), 0.0, 0.0]],
                       dtype=torch.float64, device="cuda")
    Z = torch.tensor([1.0, -0.5, 0.25], dtype=torch.float64, device="cuda")
    st, _ = _gram_noalloc(lib, ccfg, xyz, Z, n)
    assert st == _lib.RS_ERR_OUTSIDE_BOX
    assert b"outside" in lib.rs_last_error(None)
    ctx = RSContext(ccfg)
    ctx.solve(xyz, Z, energy=True, want_potential=False)
    with pytest.raises(RSError) as ei:
        ctx.energy()
    assert ei.value.status == _lib.RS_ERR_OUTSIDE_BOX
    ctx.close()
    Zbad = torch.tensor([1.0, float("nan"), 0.25], dtype=torch.float64, device="cuda")
    xyz_in = xyz.clone()
    xyz_in[2, 0] = 0.5 * b
    st, _ = _gram_noalloc(lib, ccfg, xyz_in, Zbad, n)
    assert st == _lib.RS_ERR_OUTSIDE_BOX
    # a valid call afterwards is unaffected by the failed one (the status word is cleared)
    st, _ = _gram_noalloc(lib, ccfg, xyz_in, Z, n)
    assert st == _lib.RS_OK, lib.rs_last_error(None)


def test_noalloc_rejects_problems_above_its_scratch():
    from paper_1606_09218_gb300 import _lib, config_from_workload
    lib = _lib.load()
    cfg = dict(load_config("c3_nacl28_n1025"))        # n = 1025 needs more than 16 MiB
    ccfg = config_from_workload(cfg, max_particles=4)
    xyz = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    Z = torch.ones(4, dtype=torch.float64, device="cuda")
    st, _ = _gram_noalloc(lib, ccfg, xyz, Z, 5)
    assert st == _lib.RS_ERR_CAPACITY
    assert b"16 MiB" in lib.rs_last_error(None)
