"""Spatial decomposition of one film over CPU ranks (gloo, world sizes 2 and 4): the ghost
selection, the two halo exchanges per step (positions after the drift, F'(rho) and M'(P)
after the density pass, in place of the paper's two Allgathervs, Sec. 3.3.2) and the
migration at list rebuilds of paper_1507_07068_gb300.decomp, with the FP64 oracle as every
rank's engine, against the oracle's run of the whole film."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

SKIN = 0.3
STEPS = 60


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def film():
    import md_inputs as mi
    # 12 x 12 x 6 cells, periodic x, y; the indenter over the film's centre (the corner of
    # four bricks in a 2 x 2 grid), coming down at 20 m/s; 600 K so that lists are rebuilt
    return mi.make_replica("decomp", 12, 12, 6, 6.0, 600.0, seed=77, gap=1.5)


def _forces(pot, grid, halo, x_own, xc, rank, reach):
    """One rank's Task 4: exchange 1 (ghost positions), the density pass, exchange 2 (the
    ghosts' F'(rho), M'(P) from their owners), the force pass; forces and per-atom energies
    of the owned atoms."""
    import oracle
    lo, hi, per = grid.local_box(rank, reach)
    xg = halo.positions(x_own)
    xl = np.concatenate([x_own, xg])
    n = len(x_own)
    p1 = oracle.forces_given(pot, xl, lo, hi, per, xc)
    fm = np.concatenate([p1["fm"][:n], halo.values(p1["fm"][:n])])
    given = np.r_[np.zeros(n, np.uint8), np.ones(len(xg), np.uint8)]
    p2 = oracle.forces_given(pot, xl, lo, hi, per, xc, given=given, fm_in=fm)
    return p2["F"][:n], p2["e_atom"][:n], len(xg)


def _rank_main(rank, world, port, shape, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    from paper_1507_07068_gb300 import decomp
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.set_threads(1)
        params = oracle.load_params()
        pot = oracle.Potential(params)
        rep = film()
        grid = decomp.BrickGrid(rep.box_lo, rep.box_hi, rep.periodic, shape[0], shape[1], params["rc"] + SKIN)
        ex = decomp.Exchange(dist, rank, world)
        reach = params["rc_m"] + SKIN
        mine = grid.owner(rep.x_cr) == rank
        ids = np.nonzero(mine)[0]
        x, v, fixed = rep.x_cr[mine], rep.v_cr[mine], rep.fixed[mine]
        ids, (x, v, fixed) = decomp.migrate(grid, ex, ids, [x, v, fixed])
        z, z_build = rep.z_indenter0, rep.z_indenter0
        halo = decomp.Halo(grid, ex, x)
        F, ea, ng = _forces(pot, grid, halo, x, rep.x_c + np.array([0.0, 0.0, z]), rank, reach)
        F0 = (ids.copy(), F.copy())
        xb = x.copy()
        c = 9.6485332e-3 / rep.mass_cr
        rebuilds, moved = 0, 0
        for _ in range(STEPS):
            # Task 1: the displacement rule over all ranks; migration and new ghost sets
            d = np.sqrt(((x - xb) ** 2).sum(1)).max() if len(x) else 0.0
            dmax = ex.max(d)
            if 2.0 * dmax > SKIN or dmax + abs(z - z_build) > SKIN:
                own0 = set(ids.tolist())
                ids, (x, v, F, fixed) = decomp.migrate(grid, ex, ids, [x, v, F, fixed])
                moved += len(set(ids.tolist()) ^ own0)
                halo = decomp.Halo(grid, ex, x)
                xb, z_build = x.copy(), z
                rebuilds += 1
            z += rep.v_indenter * rep.dt                                  # Task 2
            mob = fixed == 0                                              # Task 3
            v[mob] += 0.5 * rep.dt * c * F[mob]
            x[mob] += rep.dt * v[mob]
            F, ea, ng = _forces(pot, grid, halo, x, rep.x_c + np.array([0.0, 0.0, z]), rank, reach)   # Task 4
            v[mob] += 0.5 * rep.dt * c * F[mob]                           # Task 5
        epot = ex.sum([ea.sum()])[0]
        out[rank] = dict(F0=F0, ids=ids, x=x, v=v, epot=epot, rebuilds=rebuilds, moved=moved, ghosts=ng,
                         z=z)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("shape", [(2, 1), (2, 2)])
def test_decomposed_film_follows_the_single_domain_oracle(shape):
    import oracle
    from gpu_helpers import rel_force_err
    world = shape[0] * shape[1]
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), shape, out), nprocs=world, start_method="spawn",
                       join=True)
    res = [out[r] for r in range(world)]
    rep = film()
    n = rep.n_cr
    params = oracle.load_params()
    pot = oracle.Potential(params)
    # every atom owned by exactly one rank, before and after the run
    for key in ("F0", "ids"):
        got = np.concatenate([r[key][0] if key == "F0" else r[key] for r in res])
        assert np.array_equal(np.sort(got), np.arange(n))
    assert all(r["ghosts"] > 0 for r in res)
    # t = 0: forces from the two exchanges equal the whole film's
    F0 = np.zeros((n, 3))
    for r in res:
        F0[r["F0"][0]] = r["F0"][1]
    ref = oracle.forces(pot, rep.x_cr, rep.box_lo, rep.box_hi, rep.periodic, rep.x_c)
    assert rel_force_err(F0, ref["F"]).max() <= 1e-12
    # the run: same rebuild schedule, atoms migrated, trajectory and energy of the oracle's
    osim = oracle.Sim(pot, rep, skin=SKIN)
    osim.step(STEPS)
    o = osim.state()
    x = np.zeros((n, 3)); v = np.zeros((n, 3))
    for r in res:
        x[r["ids"]] = r["x"]; v[r["ids"]] = r["v"]
    assert res[0]["rebuilds"] == o["rebuilds"] > 0
    assert sum(r["moved"] for r in res) > 0
    d = x - o["x"]
    L = rep.box_hi - rep.box_lo
    d -= np.round(d / L) * L * (rep.periodic == 1)
    assert np.abs(d).max() < 1e-10
    assert np.abs(v - o["v"]).max() < 1e-12
    assert res[0]["z"] == o["z_ind"]
    assert res[0]["epot"] == pytest.approx(o["potential"], abs=1e-9 * n)
