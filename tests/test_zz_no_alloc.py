"""md_forces_small, the entry point that allocates nothing, against the existing path
(md_init + md_compute_forces in FP64 with the analytic forms) on the same systems, through
the C ABI; two calls in a row on one stream, each compared with its reference.  Also
against the FP64 oracle directly, and the device's free memory across many calls."""
import numpy as np
import pytest

import md_inputs as mi
import oracle
from gpu_helpers import jitter, rel_force_err, tiny

pytestmark = pytest.mark.gpu

TOL = 1e-12          # per-atom force bar of the FP64 path
ETOL = 1e-12         # relative bar on each energy term


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1507_07068_gb300 import md
    md.lib()
    return torch, md


def reference(md, params, rep):
    sim = md.MD([rep], params, precision="fp64", tabulated=0)
    F = sim.forces(0)
    e = sim.energy(0)
    sim.close()
    return F, e


def device_inputs(torch, rep):
    x = torch.tensor(np.ascontiguousarray(rep.x_cr), dtype=torch.float64, device="cuda")
    xc = None
    if rep.n_c:
        xc = torch.tensor(np.ascontiguousarray(rep.x_c + np.array([0.0, 0.0, rep.z_indenter0])),
                          dtype=torch.float64, device="cuda")
    F = torch.full_like(x, float("nan"))
    E = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    return x, xc, F, E


def call(md, torch, p, rep, x, xc, F, E):
    md.md_forces_small(p, rep.n_cr, x.data_ptr(), rep.n_c, xc.data_ptr() if xc is not None else None,
                       rep.box_lo, rep.box_hi, rep.periodic, F.data_ptr(), E.data_ptr(),
                       torch.cuda.current_stream().cuda_stream)


def check(F, E, ref):
    Fr, er = ref
    assert rel_force_err(F.cpu().numpy(), Fr).max() <= TOL
    e = E.cpu().numpy()
    for k, name in enumerate(("embed", "pair", "mterm", "morse")):
        assert e[k] == pytest.approx(er[name], rel=ETOL, abs=1e-12), name


def test_two_calls_in_a_row_match_the_existing_path(env, params):
    torch, md = env
    p = md.make_params(params, tabulated=0)
    md.md_forces_small(p, 0, None, 0, None, [0, 0, 0], [1, 1, 1], [0, 0, 0], None, None,
                       torch.cuda.current_stream().cuda_stream)          # set-up only
    a = tiny(amp=0.12, gap=1.0)                                           # film + indenter, periodic x, y
    b = jitter(mi.small_cluster(n_side=7, jitter=0.0, seed=5), 0.15, 5)  # free cluster, no indenter
    assert a.n_c > 0 and b.n_c == 0 and a.n_cr != b.n_cr
    ra, rb = reference(md, params, a), reference(md, params, b)
    ia, ib = device_inputs(torch, a), device_inputs(torch, b)
    call(md, torch, p, a, *ia)
    call(md, torch, p, b, *ib)
    torch.cuda.synchronize()
    check(ia[2], ia[3], ra)
    check(ib[2], ib[3], rb)
    # the same system again after a different one: nothing carried over in the scratch
    call(md, torch, p, a, *ia)
    torch.cuda.synchronize()
    check(ia[2], ia[3], ra)


def test_sizes_beyond_the_scratch_are_rejected(env, params):
    torch, md = env
    p = md.make_params(params, tabulated=0)
    n = md.MD_SMALL_MAX_ATOMS + 1
    with pytest.raises(md.MDError) as ei:
        md.md_forces_small(p, n, None, 0, None, [0, 0, 0], [50, 50, 50], [0, 0, 0], None, None, 0)
    assert ei.value.code == md.MD_ERR_ARG
    assert str(md.MD_SMALL_MAX_ATOMS) in str(ei.value)
    with pytest.raises(md.MDError) as ei:
        md.md_forces_small(md.make_params(params, tabulated=1), 10, None, 0, None, [0, 0, 0], [50, 50, 50],
                           [0, 0, 0], None, None, 0)
    assert ei.value.code == md.MD_ERR_ARG


def test_matches_the_oracle_directly(env, params):
    """The all-pairs minimum image of md_forces_small (d - L rint(d / L)) against the
    oracle's own forces and energies for a film with the indenter in reach."""
    torch, md = env
    p = md.make_params(params, tabulated=0)
    rep = tiny(amp=0.12, gap=1.0, seed=21)
    x, xc, F, E = device_inputs(torch, rep)
    call(md, torch, p, rep, x, xc, F, E)
    torch.cuda.synchronize()
    o = oracle.forces(oracle.Potential(params, tabulated=0), rep.x_cr, rep.box_lo, rep.box_hi, rep.periodic,
                      rep.x_c + np.array([0.0, 0.0, rep.z_indenter0]))
    assert rel_force_err(F.cpu().numpy(), o["F"]).max() <= TOL
    e = E.cpu().numpy()
    for k, name in enumerate(("embed", "pair", "mterm", "morse")):
        assert e[k] == pytest.approx(o[name], rel=ETOL, abs=1e-12), name


def test_no_device_memory_taken_after_set_up(env, params):
    """After the per-device set-up, calls leave the device's free memory unchanged (the
    scratch is the library's static array; nothing is allocated per call)."""
    torch, md = env
    p = md.make_params(params, tabulated=0)
    rep = tiny(amp=0.1, gap=1.5, seed=22)
    x, xc, F, E = device_inputs(torch, rep)
    stream = torch.cuda.current_stream().cuda_stream
    md.md_forces_small(p, 0, None, 0, None, [0, 0, 0], [1, 1, 1], [0, 0, 0], None, None, stream)
    call(md, torch, p, rep, x, xc, F, E)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(200):
        call(md, torch, p, rep, x, xc, F, E)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
