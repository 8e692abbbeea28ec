"""One lattice (D2Q9, or a D3Q19 box) split into x-slabs with a face
exchange after every update: the domain decomposition behind the multi-GPU
extension the paper names as future work (Sec. 6).

Each slab owns a run of whole columns (planes in 3-D) and adds one ghost
column on every face it shares with another slab. The pull update (Eq. 1) of
a slab's boundary column reads, from the ghost column beside it, only the
populations that cross that face (three per node in D2Q9, five in D3Q19);
after every update the owner of the neighbouring column sends exactly those
(``lbm_face_pack``) and the slab writes them into its ghost column
(``lbm_face_unpack``). Solid padding columns beyond a ghost column can round
a slab's row length up to a multiple of 32 nodes, so that its rows keep the
memory-line alignment of the undivided lattice's. With the ghost columns'
solid mask taken from the neighbour, every interior node sees the same
sources, the same link classification and the same edge treatment as in the
undivided lattice, so the interiors evolve bit for bit like it (LPTL, NPTL,
NPOL, NSOL; every layout and storage; stochastic rounding keys its draws on
each slab's own node index, so it gives other, equally distributed, draws).
The ghost columns' own updates are never read and are overwritten by the
next exchange.

Two transports carry a face's message:
 * slabs held by the same process exchange on the device, every message of
   an update in one launch (``lbm_face_exchange``: column to ghost column,
   no buffer; one stream, so no synchronisation);
 * slabs held by different processes exchange through page-locked host
   buffers over a ``torch.distributed`` process group (one slab per rank,
   slab index = rank): device -> host copy, point-to-point send/recv with the
   face's two neighbours, host -> device copy, unpack.

Every step of the update and of the exchange runs in the library's kernels;
this module only plans the split and moves the messages.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import lbm

ELEM_BYTES = {"f64": 8, "f32": 4, "f16s": 2, "bf16s": 2}
EAST_GOING, WEST_GOING = 1, -1   # sense: c_ix of the exchanged directions


@dataclass(frozen=True)
class Slab:
    """Columns [x0, x1) of the lattice, plus a ghost column on the west
    (gw = 1) and / or east (ge = 1) face, and pw / pe solid padding columns
    outside the ghost columns that round the slab's row length up to the
    alignment asked for. Local columns, west to east: pw padding, gw ghost,
    the interior, ge ghost, pe padding."""
    index: int
    x0: int
    x1: int
    gw: int
    ge: int
    pw: int = 0
    pe: int = 0

    @property
    def width(self) -> int:
        return self.x1 - self.x0

    @property
    def nx(self) -> int:
        """Columns of the slab's own lattice, ghosts and padding included."""
        return self.pw + self.gw + self.width + self.ge + self.pe

    @property
    def first(self) -> int:
        """Local column of the first interior column."""
        return self.pw + self.gw

    @property
    def interior(self) -> slice:
        return slice(self.first, self.first + self.width)

    @property
    def west_ghost(self) -> int:
        return self.pw

    @property
    def east_ghost(self) -> int:
        return self.first + self.width

    def columns(self, nx: int) -> np.ndarray:
        """Lattice column held by each ghost and interior column of the slab
        (ghosts wrap on a periodic lattice)."""
        return np.arange(self.x0 - self.gw, self.x1 + self.ge) % nx

    def local(self, a: np.ndarray, nx: int, pad_value) -> np.ndarray:
        """The slab's columns of a lattice array (ny x nx, y-major), padding
        columns filled with pad_value."""
        a = np.asarray(a).reshape(-1, nx)
        out = np.full((a.shape[0], self.nx), pad_value, a.dtype)
        out[:, self.pw:self.nx - self.pe] = a[:, self.columns(nx)]
        return out

    def edges(self, bc) -> tuple:
        """(west, east, south, north) of the slab's lattice: the lattice's own
        x edge where the slab has no ghost column, a wall beyond a ghost or a
        padding column (only the ghost's own update, never read, sees it)."""
        return (lbm.WALL if (self.gw or self.pw) else bc[0], lbm.WALL if (self.ge or self.pe) else bc[1],
                bc[2], bc[3])


def split(nx: int, parts: int, periodic_x: bool, align: int = 1) -> list[Slab]:
    """Columns split into `parts` runs whose widths differ by at most one.
    Every slab holds at least two columns, so the column next to an inlet or
    outlet edge (read by the Neumann inlet) is never a ghost. With align > 1
    a slab with a ghost column gets solid padding beyond it (east if it has
    an east ghost, else west) so that its row length is a multiple of align:
    rows then start on the same memory-line boundary as an undivided
    lattice's."""
    if parts < 1 or 2 * parts > nx:
        raise ValueError(f"cannot split {nx} columns into {parts} slabs of at least 2 columns")
    if align < 1:
        raise ValueError("align must be >= 1")
    base, extra = divmod(nx, parts)
    wrap = periodic_x and parts > 1
    out, x = [], 0
    for s in range(parts):
        w = base + (1 if s < extra else 0)
        gw, ge = 1 if (s > 0 or wrap) else 0, 1 if (s < parts - 1 or wrap) else 0
        pad = (-(gw + w + ge)) % align if (gw or ge) else 0
        out.append(Slab(s, x, x + w, gw, ge, 0 if ge else pad, pad if ge else 0))
        x += w
    return out


def faces(parts: int, periodic_x: bool) -> list[tuple[int, int]]:
    """Shared faces as (west slab, east slab) pairs."""
    f = [(s, s + 1) for s in range(parts - 1)]
    if periodic_x and parts > 1:
        f.append((parts - 1, 0))
    return f


def messages(slabs: list[Slab], periodic_x: bool) -> list[tuple[int, int, int, int, int]]:
    """Per update, every message as (sender, column in sender, receiver,
    column in receiver, sense): across each face the west slab's last
    interior column sends its east-going populations into the east slab's
    west ghost, and the east slab's first interior column sends its
    west-going populations into the west slab's east ghost."""
    out = []
    for w, e in faces(len(slabs), periodic_x):
        sw, se = slabs[w], slabs[e]
        out.append((w, sw.east_ghost - 1, e, se.west_ghost, EAST_GOING))
        out.append((e, se.first, w, sw.east_ghost, WEST_GOING))
    return out


def _tag(sense: int) -> int:
    return 0 if sense == EAST_GOING else 1


def exchange_host(sends: list, recvs: list, group=None):
    """Point-to-point exchange of host buffers over a torch.distributed group:
    sends / recvs are lists of (peer, sense, tensor), peer = the other slab's
    index = its rank in `group` (default: the world). Messages between the
    same two ranks are told apart by their sense (two of them when two slabs
    share both faces of a periodic lattice). All receives are posted before
    the sends, and every request is waited for."""
    import torch.distributed as dist
    g = (lambda r: r) if group is None else (lambda r: dist.get_global_rank(group, r))
    reqs = [dist.irecv(t, src=g(peer), group=group, tag=_tag(sense)) for peer, sense, t in recvs]
    reqs += [dist.isend(t, dst=g(peer), group=group, tag=_tag(sense)) for peer, sense, t in sends]
    for r in reqs:
        r.wait()


def edges3(sl: Slab, bc, bc_x_east: int) -> tuple:
    """(bc_x, bc_y, bc_z, bc_x_east) of a D3Q19 slab's box: the box's own
    x faces where the slab has no ghost plane; walls beyond ghost or padding
    planes of a periodic or walled box; the box's inlet / outlet pair
    otherwise, applied to the slab's end planes (a ghost or padding plane
    there only changes that plane's own update, which is never read: the
    inlet and outlet treatments read and write the node itself)."""
    if not (sl.gw or sl.ge) or bc[0] not in (lbm.PERIODIC, lbm.WALL):
        return bc[0], bc[1], bc[2], bc_x_east
    return lbm.WALL, bc[1], bc[2], bc_x_east


class Decomposition:
    """A lattice of nx x ny nodes (D2Q9), or nx x ny x nz (D3Q19, with nz),
    split into `parts` x-slabs.

    owned: slab indices held by this process, one lattice each on the current
    device (default: all). When some slabs live elsewhere, slab s is held by
    rank s of `group` (a torch.distributed process group, default the world)
    and their faces exchange through host memory. align: row length of
    every slab's lattice rounded up to a multiple of this many nodes with
    solid padding (1 = none). Other keyword arguments are those of
    ``lbm.Lattice`` or ``lbm.Lattice3`` (bc, layout, algo, storage, force,
    ...); in 3-D bc = (x, y, z) and bc_x_east as for ``lbm.Lattice3``."""

    def __init__(self, nx, ny, tau, mask=None, *, nz=None, parts=2, owned=None, group=None, bc=None,
                 align=32, **kw):
        import torch
        algo = kw.get("algo", "nptl")
        if (lbm.ALGOS[algo] if isinstance(algo, str) else int(algo)) == lbm.ALGOS["aa"]:
            raise ValueError("the AA pattern stores two forms of the state in turn; slabs need one")
        self.d3 = nz is not None
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz) if self.d3 else 1
        self.rows = self.ny * self.nz
        if bc is None:
            bc = (lbm.PERIODIC,) * (3 if self.d3 else 4)
        self.periodic_x = bc[0] == lbm.PERIODIC and (self.d3 or bc[1] == lbm.PERIODIC)
        self.slabs = split(self.nx, int(parts), self.periodic_x, int(align))
        self.owned = list(range(len(self.slabs))) if owned is None else sorted(int(s) for s in owned)
        self.group = group
        storage = kw.get("storage", "f32")
        storage = storage if isinstance(storage, str) else {v: k for k, v in lbm.STORAGES.items()}[storage]
        self.elem = ELEM_BYTES[storage]
        self.q = 19 if self.d3 else 9
        m = np.zeros((self.rows, self.nx), np.uint8) if mask is None else \
            np.asarray(mask, np.uint8).reshape(self.rows, self.nx)
        bc_x_east = kw.pop("bc_x_east", lbm.OUTFLOW_ZG)
        self.lat = {}
        for s in self.owned:
            sl = self.slabs[s]
            local = sl.local(m, self.nx, 1)
            if self.d3:
                bx, by, bz, bxe = edges3(sl, bc, bc_x_east)
                self.lat[s] = lbm.Lattice3(sl.nx, self.ny, self.nz, tau, local, bc=(bx, by, bz), bc_x_east=bxe,
                                           **kw)
            else:
                self.lat[s] = lbm.Lattice(sl.nx, self.ny, tau, local, bc=sl.edges(bc), **kw)
        self.msgs = messages(self.slabs, self.periodic_x)
        nb = (5 if self.d3 else 3) * self.rows * self.elem
        dev = lambda: torch.empty(nb, dtype=torch.uint8, device="cuda")  # noqa: E731
        host = lambda: torch.empty(nb, dtype=torch.uint8, pin_memory=True)  # noqa: E731
        # buffers for messages to or from another process only (the others go column to column)
        remote = [k for k, (src, _, dst, _, _) in enumerate(self.msgs) if (src in self.lat) != (dst in self.lat)]
        self.dbuf = {k: dev() for k in remote}
        self.hbuf = {k: host() for k in remote}

    def _field(self, a, sl: Slab):
        if a is None:
            return None
        return sl.local(np.asarray(a, np.float64), self.nx, 0.0).reshape(-1)

    def init(self, rho=None, ux=None, uy=None, uz=None):
        """Equilibrium from the lattice's fields (N values each, x fastest);
        every slab, ghost columns included, starts from the same state as the
        undivided lattice, so the first update needs no exchange."""
        for s, lat in self.lat.items():
            f = [self._field(a, self.slabs[s]) for a in ((rho, ux, uy, uz) if self.d3 else (rho, ux, uy))]
            lat.init(*f)
        return self

    def exchange(self):
        import torch
        local = [m for m in self.msgs if m[0] in self.lat and m[2] in self.lat]
        if local:
            src, xs, dst, xd, sense = zip(*local)
            fn = lbm.lbm3_face_exchange if self.d3 else lbm.lbm_face_exchange
            fn([self.lat[s].h for s in src], xs, [self.lat[d].h for d in dst], xd, sense, self.lat[src[0]].stream)
        sends, recvs = [], []
        for k in self.dbuf:  # messages to or from another process
            src, xs, dst, xd, sense = self.msgs[k]
            if src in self.lat:
                lat = self.lat[src]
                lat.face_pack(xs, sense, self.dbuf[k])
                with torch.cuda.stream(lat.torch_stream):
                    self.hbuf[k].copy_(self.dbuf[k], non_blocking=True)
                sends.append((dst, sense, self.hbuf[k]))
            else:
                recvs.append((src, sense, self.hbuf[k]))
        if not self.dbuf:
            return
        for lat in self.lat.values():
            lat.sync()  # packed messages in host memory, receivers' updates done
        exchange_host(sends, recvs, self.group)
        for k in self.dbuf:
            src, xs, dst, xd, sense = self.msgs[k]
            if dst in self.lat:
                lat = self.lat[dst]
                with torch.cuda.stream(lat.torch_stream):
                    self.dbuf[k].copy_(self.hbuf[k], non_blocking=True)
                lat.face_unpack(xd, sense, self.dbuf[k])

    def step(self, n: int = 1, moments: bool = False):
        for t in range(int(n)):
            last = moments and t == n - 1
            for lat in self.lat.values():
                lat.step(1, moments=last)
            self.exchange()
        return self

    def sync(self):
        for lat in self.lat.values():
            lat.sync()
        return self

    def _assemble(self, parts: dict, lead: int | None):
        shape = (self.rows, self.nx) if lead is None else (lead, self.rows, self.nx)
        out = None
        for s, a in parts.items():
            sl = self.slabs[s]
            a = a.reshape(shape[:-1] + (sl.nx,))[..., sl.interior]
            if out is None:
                out = np.zeros(shape, a.dtype)
            out[..., sl.x0:sl.x1] = a
        return out.reshape(shape[:-2] + (-1,))

    def moments(self):
        """(rho, ux, uy[, uz]) of the owned slabs' interior columns, placed
        in lattice-sized arrays (columns of slabs held elsewhere stay 0)."""
        got = {s: lat.moments() for s, lat in self.lat.items()}
        return tuple(self._assemble({s: m[c] for s, m in got.items()}, None) for c in range(4 if self.d3 else 3))

    def populations(self, as_: str = "f64") -> np.ndarray:
        """(Q, N) state of the owned slabs' interior columns (others 0)."""
        return self._assemble({s: lat.populations(as_) for s, lat in self.lat.items()}, self.q)

    def close(self):
        for lat in self.lat.values():
            lat.close()
        self.lat = {}
