"""One periodic domain split into z-slabs, one slab per handle or per rank.

The scheme moves populations only along the lattice axes (D3Q7, Sec. 2.2), so a
slab that is periodic in z on its own differs from its part of the whole domain
only in the two z-moving populations of its boundary planes: through its own z
wrap, the bottom plane takes its +z population from its own top plane, and the
top plane its -z population from its own bottom plane. Ring shifts of one plane of
one storage slot (14 fields) per face put the neighbours' values there instead.

* Two-buffer pull stepping (the state holds f_i(x) after every step), after each
  step: the bottom plane's +z values move one slab up the ring (slab r's wrapped
  value is the one slab r+1 needs), the top plane's -z values one slab down.
* In-place AA stepping (slot i of cell x holds f_i(x) after an even number of
  steps): an even step touches only a cell's own slots, but leaves the state in
  the form where f_i(x) sits in slot opp(i) of cell x - e_i, so reads of the state
  (the next odd step's, or any output's) go through the z wrap: the bottom plane's
  +z value comes from the -z slot of the top plane, the top plane's -z value from
  the +z slot of the bottom plane. After an even step, therefore, the top planes'
  -z slots move one slab up and the bottom planes' +z slots one slab down. An odd
  step reads those slots and writes the same ones through the wrap; after it, the
  bottom planes' +z slots move up and the top planes' -z slots down, taking the
  wrapped writes to the cells they belong to.

Each exchange moves 14 * nx * ny elements per face. With one slab every shift is the
identity and the slab is the periodic domain.
"""
from __future__ import annotations

import numpy as np

PLUS_Z, MINUS_Z = 5, 6
UP, DOWN = 1, -1  # UP: slab r's plane goes to slab r + 1

PULL_AFTER_STEP = (("bottom", PLUS_Z, UP), ("top", MINUS_Z, DOWN))
AA_AFTER_EVEN = (("top", MINUS_Z, UP), ("bottom", PLUS_Z, DOWN))
AA_AFTER_ODD = (("bottom", PLUS_Z, UP), ("top", MINUS_Z, DOWN))


def slab_bounds(nz: int, parts: int) -> list[tuple[int, int]]:
    """Planes [z0, z1) of each slab: as equal as possible, the first nz % parts
    slabs one plane thicker. Every slab has at least one plane."""
    if parts < 1 or nz < parts:
        raise ValueError(f"cannot split {nz} planes into {parts} slabs")
    base, extra = divmod(nz, parts)
    out, z0 = [], 0
    for r in range(parts):
        z1 = z0 + base + (1 if r < extra else 0)
        out.append((z0, z1))
        z0 = z1
    return out


def plane_index(which: str, nz_local: int) -> int:
    return 0 if which == "bottom" else nz_local - 1


def ring_shift(items: list, shift: int) -> list:
    """out[r] = items[r - shift] (cyclic)."""
    n = len(items)
    return [items[(r - shift) % n] for r in range(n)]


def dist_ring_shift(t, shift: int, dist, group=None):
    """The ring shift across ranks: sends t to rank r + shift and returns what rank
    r - shift sent (torch.distributed point-to-point; a tensor of the same shape)."""
    world = dist.get_world_size(group)
    if world == 1:
        return t.clone()
    rank = dist.get_rank(group)
    dst, src = (rank + shift) % world, (rank - shift) % world
    out = t.new_empty(t.shape)
    reqs = [dist.isend(t.contiguous(), dst, group=group), dist.irecv(out, src, group=group)]
    for q in reqs:
        q.wait()
    return out


class SlabRing:
    """Slab handles of one domain held in one process (one device or several; planes
    move between devices as tensor copies), stepped with the AA exchanges through
    lbm_plane_get / lbm_plane_set on device buffers. The handles must share Q_ref and storage scales (e.g. FP32 or BF16
    storage initialised with lbm_init_tgv, then loaded with their part of one state)."""

    def __init__(self, domains: list):
        self.domains = list(domains)
        d0 = self.domains[0]
        for d in self.domains:
            if (d.nx, d.ny, d.store) != (d0.nx, d0.ny, d0.store):
                raise ValueError("slabs differ in nx, ny or storage")
            a, b = d.info(), d0.info()
            if (a["rho_ref"], a["E_ref"], a["scale"]) != (b["rho_ref"], b["E_ref"], b["scale"]):
                raise ValueError("slabs differ in Q_ref or storage scales")

    def _exchange(self, plan):
        import torch
        for which, slot, shift in plan:
            planes = [d.plane_get(plane_index(which, d.nz), slot) for d in self.domains]
            for d in self.domains:
                torch.cuda.synchronize(d.device)
            for d, buf in zip(self.domains, ring_shift(planes, shift)):
                # a plane from a slab on another device is copied to this one first
                d.plane_set(plane_index(which, d.nz), slot, buf.to(d.device))
            for d in self.domains:
                torch.cuda.synchronize(d.device)

    def step(self, n: int = 1):
        for _ in range(n):
            odd = self.domains[0].step_count & 1
            for d in self.domains:
                d.step(1)
            self._exchange(AA_AFTER_ODD if odd else AA_AFTER_EVEN)


class SlabRank:
    """This rank's slab handle in a torch.distributed job (one process per GPU),
    stepped with the AA exchanges. staging="device" sends device tensors (NCCL);
    staging="host" goes through host memory (gloo)."""

    def __init__(self, domain, dist, group=None, staging: str = "device"):
        self.d, self.dist, self.group, self.staging = domain, dist, group, staging

    def _exchange(self, plan):
        import torch
        d = self.d
        for which, slot, shift in plan:
            z = plane_index(which, d.nz)
            if self.staging == "host":
                buf = np.empty((14, d.ny, d.nx), dtype=d.plane_dtype(numpy=True))
                d.plane_get(z, slot, buf)
                got = dist_ring_shift(torch.from_numpy(buf), shift, self.dist, self.group)
                d.plane_set(z, slot, got.numpy())
            else:
                buf = d.plane_get(z, slot)
                torch.cuda.synchronize(d.device)
                got = dist_ring_shift(buf, shift, self.dist, self.group)
                d.plane_set(z, slot, got)

    def step(self, n: int = 1):
        for _ in range(n):
            odd = self.d.step_count & 1
            self.d.step(1)
            self._exchange(AA_AFTER_ODD if odd else AA_AFTER_EVEN)
