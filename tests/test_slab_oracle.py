"""z-slab decomposition on CPU ranks (gloo): the FP64 oracle split into slabs, each
periodic in z on its own, with the ring exchanges of slab.py after every step, must
give the single-domain oracle's populations bit for bit; world sizes 2 and 3 (uneven
slabs). Also the slab bounds and ring shifts themselves."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

from conftest import ROOT, make_oracle

NX, NY, NZ, STEPS = 8, 6, 10, 9


def _params():
    from paper_2608_13437_gb300 import inputs
    p = inputs.tgv_params(8)
    p.update(nx=NX, ny=NY, nz=NZ, sutherland=0, f_mu=0.3, J_min=1e-3, tau_R=0.05, tau_q=0.05)
    return p


def _fields():
    from paper_2608_13437_gb300 import inputs
    return inputs.random_smooth_state(NX, NY, NZ, seed=37, amp=0.15)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as dist
    from conftest import make_oracle as mk
    from oracle import oracle as orc
    from paper_2608_13437_gb300 import slab
    orc.set_threads(1)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    z0, z1 = slab.slab_bounds(NZ, world)[rank]
    p = dict(_params(), nz=z1 - z0)
    s = _fields()
    o = mk(p)
    o.init_fields(*[s[k][z0:z1] for k in ("rho", "ux", "uy", "uz", "p")])
    for _ in range(STEPS):
        o.step(1)
        f = o.populations()
        for which, sl, shift in slab.PULL_AFTER_STEP:
            zi = slab.plane_index(which, z1 - z0)
            got = slab.dist_ring_shift(torch.from_numpy(f[:, sl, zi].copy()), shift, dist)
            f[:, sl, zi] = got.numpy()
        o.set_populations(f)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, z0, z1, o.populations()))


@pytest.mark.parametrize("world", [2, 3])
def test_oracle_slabs_on_gloo_ranks_equal_one_domain(world, oracle_mod):
    pytest.importorskip("torch")
    whole = make_oracle(_params())
    s = _fields()
    whole.init_fields(s["rho"], s["ux"], s["uy"], s["uz"], s["p"])
    whole.step(STEPS)
    ref = whole.populations()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, z0, z1, f in res:
        assert np.array_equal(f, ref[:, :, z0:z1]), rank
    # without the exchanges the slabs would not match (the test can fail)
    lone = make_oracle(dict(_params(), nz=NZ // 2))
    lone.init_fields(*[s[k][:NZ // 2] for k in ("rho", "ux", "uy", "uz", "p")])
    lone.step(STEPS)
    assert not np.array_equal(lone.populations(), ref[:, :, :NZ // 2])


def test_slab_bounds_and_ring_shift():
    from paper_2608_13437_gb300 import slab
    assert slab.slab_bounds(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert slab.slab_bounds(4, 4) == [(0, 1), (1, 2), (2, 3), (3, 4)]
    assert slab.slab_bounds(7, 1) == [(0, 7)]
    with pytest.raises(ValueError):
        slab.slab_bounds(2, 3)
    assert slab.ring_shift([0, 1, 2], slab.UP) == [2, 0, 1]
    assert slab.ring_shift([0, 1, 2], slab.DOWN) == [1, 2, 0]
    assert slab.ring_shift(["a"], slab.UP) == ["a"]
    # the exchanges after even and after odd steps touch the same (plane, slot) pairs
    assert {(w, s) for w, s, _ in slab.AA_AFTER_EVEN} == {(w, s) for w, s, _ in slab.AA_AFTER_ODD}
    assert slab.AA_AFTER_ODD == slab.PULL_AFTER_STEP


# In-place AA stepping emulated in numpy on one field with a nonlinear cell-local map:
# the same index maps as the GPU kernel (even: own slots in, opposite slots out; odd:
# slot opp(i) of x - e_i in, slot i of x + e_i out).
OPP = (0, 2, 1, 4, 3, 6, 5)
E = ((0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))


def _roll(a, e):  # value at x comes from x - e; arrays are [z][y][x]
    return np.roll(a, shift=(e[2], e[1], e[0]), axis=(0, 1, 2))


def _cell_map(f):
    s = f.sum(axis=0)
    return np.stack([f[i] + 0.3 * (s / 7 - f[i]) + 0.05 * np.sin((i + 1) * f[i] + s) for i in range(7)])


def _aa_step(arr, odd):
    if not odd:
        post = _cell_map(arr)
        return np.stack([post[OPP[i]] for i in range(7)])
    pre = np.stack([_roll(arr[OPP[i]], E[i]) for i in range(7)])
    post = _cell_map(pre)
    return np.stack([_roll(post[i], E[i]) for i in range(7)])


def _canonical(arr, odd):
    return np.stack([_roll(arr[OPP[i]], E[i]) for i in range(7)]) if odd else arr.copy()


@pytest.mark.parametrize("parts", [1, 2, 3, 7])
def test_aa_slab_exchanges_reproduce_the_whole_domain(parts):
    """slab.py's exchanges after even and after odd steps make slab-periodic in-place
    (AA) stepping equal the whole periodic domain after every step."""
    from paper_2608_13437_gb300 import slab
    rng = np.random.default_rng(5)
    nz = 7
    whole = rng.standard_normal((7, nz, 5, 6))
    bounds = slab.slab_bounds(nz, parts)
    slabs = [whole[:, z0:z1].copy() for z0, z1 in bounds]
    for step in range(6):
        odd = step & 1
        whole = _aa_step(whole, odd)
        slabs = [_aa_step(a, odd) for a in slabs]
        for which, sl, shift in (slab.AA_AFTER_ODD if odd else slab.AA_AFTER_EVEN):
            planes = [a[sl, slab.plane_index(which, a.shape[1])].copy() for a in slabs]
            for a, pl in zip(slabs, slab.ring_shift(planes, shift)):
                a[sl, slab.plane_index(which, a.shape[1])] = pl
        ref = _canonical(whole, not odd)
        for (z0, z1), a in zip(bounds, slabs):
            assert np.array_equal(_canonical(a, not odd), ref[:, z0:z1]), (step, z0)

