"""z-slab decomposition of one domain on the GPU: slab handles, each periodic in z on
its own, stepped with the AA exchanges of slab.py through lbm_plane_get /
lbm_plane_set, equal the whole domain bit for bit. In one process (SlabRing: several
handles on one GPU) and as two gloo ranks sharing the GPU that exchange through host
memory (SlabRank). No kernel waits on another: the host orders every exchange."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

from conftest import ROOT
from paper_2608_13437_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_13437_gb300 import build, lbm as L
    build.build()
    L.lib()
    return L


def _params(case):
    if case == "tgv32":
        return inputs.tgv_params(32)
    # ragged: rows of 48 cells, so tiles of 32 cells straddle rows; still a periodic
    # TGV (three periods along x)
    p = inputs.tgv_params(16)
    p.update(nx=48)
    return p


def _slabs(lbm, p, store, bounds, f_native):
    out = []
    for z0, z1 in bounds:
        d = lbm.Domain(dict(p, nz=z1 - z0), store=store)
        d.init_tgv(1.0, 1.25, 1.0)  # the same Q_ref as the whole domain
        d.set_populations(np.ascontiguousarray(f_native[:, :, z0:z1]), native=True)
        out.append(d)
    return out


def _bits(f):
    return f.view(np.uint32) if f.dtype == np.float32 else f


@pytest.mark.parametrize("case,store,parts,steps", [("tgv32", "f32", 3, 7), ("ragged", "bf16", 2, 9),
                                                    ("ragged", "f32", 16, 4), ("ragged", "f32", 5, 6)])
def test_slab_ring_equals_whole_domain(lbm, case, store, parts, steps):
    from paper_2608_13437_gb300 import slab
    p = _params(case)
    whole = lbm.Domain(p, store=store)
    whole.init_tgv(1.0, 1.25, 1.0)
    f0 = whole.populations("native")
    bounds = slab.slab_bounds(p["nz"], parts)
    ring = slab.SlabRing(_slabs(lbm, p, store, bounds, f0))
    whole.step(steps)
    ring.step(steps)
    f = whole.populations("native")
    assert np.isfinite(whole.populations()).all()
    for (z0, z1), d in zip(bounds, ring.domains):
        assert d.step_count == steps
        assert np.array_equal(_bits(d.populations("native")), _bits(f[:, :, z0:z1])), (z0, z1)
    # control: the same slabs without the exchanges do not match
    lone = _slabs(lbm, p, store, bounds, f0)
    for d in lone:
        d.step(steps)
    assert not all(np.array_equal(_bits(d.populations("native")), _bits(f[:, :, z0:z1]))
                   for (z0, z1), d in zip(bounds, lone))
    for d in ring.domains + lone + [whole]:
        d.close()


def test_plane_get_set_round_trip_and_errors(lbm):
    from paper_2608_13437_gb300 import slab
    p = _params("ragged")
    d = lbm.Domain(p, store="bf16")
    d.init_tgv(1.0, 1.25, 1.0)
    d.step(3)
    f = d.populations("native")  # odd parity: canonical order differs from storage slots
    host = np.empty((14, 16, 48), dtype=np.int16)
    d.plane_get(4, slab.PLUS_Z, host)
    dev = d.plane_get(4, slab.PLUS_Z)
    assert np.array_equal(dev.cpu().numpy(), host)
    d.plane_set(2, slab.MINUS_Z, host)
    assert np.array_equal(d.plane_get(2, slab.MINUS_Z).cpu().numpy(), host)
    d.plane_set(2, slab.MINUS_Z, dev.new_zeros(dev.shape))
    g = d.populations("native")
    assert not np.array_equal(f, g)  # the write landed in the state
    for z, s in ((-1, 5), (16, 5), (0, 7), (0, -1)):
        with pytest.raises(lbm.LbmError) as ei:
            d.plane_get(z, s, host)
        assert ei.value.status == lbm.LBM_E_INVAL
    d.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, case, store, steps, f0, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2608_13437_gb300 import lbm as L, slab
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = _params(case)
    z0, z1 = slab.slab_bounds(p["nz"], world)[rank]
    d = _slabs(L, p, store, [(z0, z1)], f0)[0]
    slab.SlabRank(d, dist, staging="host").step(steps)
    out = d.populations("native")
    d.close()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, z0, z1, out))


def test_slab_ranks_over_gloo_equal_whole_domain(lbm):
    p = _params("tgv32")
    whole = lbm.Domain(p)
    whole.init_tgv(1.0, 1.25, 1.0)
    f0 = whole.populations("native")
    whole.step(5)
    f = whole.populations("native")
    whole.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, "tgv32", "f32", 5, f0, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=300) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank, z0, z1, out in res:
        assert np.array_equal(_bits(out), _bits(f[:, :, z0:z1])), rank
