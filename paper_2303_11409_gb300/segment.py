"""Chain segmentation: one TEBD chain split into contiguous segments, one per rank.

Sec. II of arXiv:2303.11409 processes independent two-site updates in parallel and
distributes the work across GPUs and nodes.  Here a chain of L sites is cut at even
site indices 0 = b_0 < b_1 < ... < b_R = L; rank r owns the sites [b_r, b_{r+1}).  With
the Strang schedule the odd layers (left sites 0, 2, 4, ...) never straddle a cut and
run locally.  An even layer (left sites 1, 3, 5, ...) has one update per cut, on the
sites (b_r - 1, b_r): both neighbouring ranks compute it, from the same inputs, with
the same kernels, so they get the same result bit for bit, and each keeps the part it
owns.  For that, each rank holds a ghost copy of the site just outside each end of its
segment, refreshed by one exchange before every layer that has straddling updates:
rank r sends its first owned site (with the charge table and Schmidt values of the bond
right of it) to rank r-1, and its last owned site (with the bond left of it) to rank
r+1.  That is the only communication; there is no reduction and no send-back.

The engine (the state and its updates) is pluggable: GpuEngine runs the CUDA library on
a handle that allocates only the owned and ghost sites (mps_create_segment); the
transport is torch.distributed point-to-point messages (NCCL between GPUs, gloo on the
host), carrying one packed float64 buffer per site.
"""
from __future__ import annotations

import numpy as np

import ctypes

from ._binding import MPS, MPS_FP64, MPSError, _default_stream, _h, _i32, _i32p, _ptr, lib


def cuts(L: int, world: int) -> list[int]:
    """Segment boundaries b_0 = 0 < ... < b_R = L, inner ones even, sizes as equal as the
    parity allows (every segment holds at least two sites)."""
    if world < 1 or L < 2 * world:
        raise ValueError("need at least two sites per rank")
    b = [0]
    for r in range(1, world):
        x = int(round(r * L / world))
        x -= x % 2
        x = max(x, b[-1] + 2)
        b.append(x)
    b.append(L)
    if any(b[i + 1] - b[i] < 2 for i in range(world)) or b[-2] >= L:
        raise ValueError("chain too short for this many ranks")
    return b


class Segment:
    """The sites a rank owns and the updates of a layer it performs."""

    def __init__(self, L: int, world: int, rank: int):
        self.L, self.world, self.rank = L, world, rank
        self.b = cuts(L, world)
        self.lo, self.hi = self.b[rank], self.b[rank + 1]

    def updates(self, sites):
        """Left sites s of the layer with (s, s+1) touching the segment: the local ones and
        the straddling ones at either cut."""
        return [s for s in sites if self.lo - 1 <= s <= self.hi - 1 and s + 1 <= self.L - 1]

    def straddles(self, sites) -> bool:
        """True when some update of the layer crosses a cut (then ghosts must be current)."""
        inner = self.b[1:-1]
        return any((c - 1) in sites for c in inner)

    def held(self):
        """Sites held on this rank: the owned ones and a ghost beyond each inner cut."""
        return max(0, self.lo - 1), min(self.L, self.hi + 1)


# ---------------------------------------------------------------------------
# packing one site and a neighbouring bond into one float64 buffer
# ---------------------------------------------------------------------------
def pack(site: int, bond: int, lam: dict, blocks: dict) -> np.ndarray:
    """[site, bond, n_sectors, charges..., dims..., lambda..., n_blocks, (l, m)...,
    block data (re, im)...] as float64 (integers are exact below 2^53)."""
    ch = sorted(lam)
    keys = sorted(blocks)
    parts = [np.array([site, bond, len(ch)], np.float64), np.array(ch, np.float64),
             np.array([len(lam[c]) for c in ch], np.float64)]
    parts += [np.asarray(lam[c], np.float64) for c in ch]
    parts.append(np.array([len(keys)], np.float64))
    parts.append(np.array([x for k in keys for x in k], np.float64))
    for k in keys:
        parts.append(np.asarray(blocks[k], np.complex128).reshape(-1).view(np.float64))
    return np.concatenate(parts)


def unpack(buf: np.ndarray):
    """Inverse of pack: (site, bond, lambda per charge, block labels, flat block data);
    place_blocks shapes the data once the dims of both bonds of the site are known."""
    site, bond, n = int(buf[0]), int(buf[1]), int(buf[2])
    o = 3
    ch = [int(x) for x in buf[o:o + n]]
    o += n
    dims = [int(x) for x in buf[o:o + n]]
    o += n
    lam = {}
    for c, k in zip(ch, dims):
        lam[c] = buf[o:o + k].copy()
        o += k
    nb = int(buf[o])
    o += 1
    pairs = [(int(buf[o + 2 * i]), int(buf[o + 2 * i + 1])) for i in range(nb)]
    o += 2 * nb
    return site, bond, lam, pairs, buf[o:]


def place_blocks(pairs, data: np.ndarray, left: dict, right: dict) -> dict:
    out, o = {}, 0
    for (l, m) in pairs:
        n = left[l] * right[m]
        out[(l, m)] = data[o:o + 2 * n].view(np.complex128).reshape(left[l], right[m]).copy()
        o += 2 * n
    return out


# ---------------------------------------------------------------------------
# engines
# ---------------------------------------------------------------------------
class GpuEngine:
    """The CUDA library on one handle that holds only this rank's sites and ghosts."""

    def __init__(self, seg: Segment, d: int, occupations, chi_max: int, precision: int = MPS_FP64, stream=None):
        lo, hi = seg.held()
        occ = _i32(occupations)
        obj = MPS.__new__(MPS)
        obj.L, obj.d, obj.chi_max = len(occ), int(d), int(chi_max)
        obj.stream = _default_stream() if stream is None else stream
        h = _h()
        rc = lib.mps_create_segment(ctypes.byref(h), obj.L, obj.d, _ptr(occ, _i32p), lo, hi, precision,
                                    obj.chi_max, obj.stream)
        if rc != 0:
            raise MPSError(rc, "mps_create_segment failed")
        obj._h = h
        obj.N = int(occ.sum())
        self.psi = obj

    def apply_layer(self, sites, gates, chi, cutoff):
        if sites:
            self.psi.apply_layer(sites, gates, chi, cutoff)

    def bond(self, b):
        return self.psi.bond(b)

    def site(self, s):
        return self.psi.site(s)

    def load(self, bond, lam, site, blocks):
        if 1 <= bond <= self.psi.L - 1:
            self.psi.set_bond(bond, lam)
        self.psi.set_site(site, blocks)

    def bond_dims(self, b):
        return self.psi.bond_dims(b)


class SegmentedTEBD:
    """Runs Strang layers of one chain split over the ranks of a torch.distributed group."""

    def __init__(self, seg: Segment, engine, dist, group=None, device=None):
        self.seg, self.engine, self.dist, self.group = seg, engine, dist, group
        self.device = device           # where the exchanged buffers live (None: host tensors, gloo)
        self.exchanges = 0

    def _send_recv(self, sends: dict, recv_from: list):
        """Point-to-point: size first, then the payload; every send is posted before the
        receives, so neighbours exchanging at the same time do not wait on one another."""
        import torch
        reqs, out = [], {}
        dev = self.device or "cpu"
        hold = []
        for peer, buf in sends.items():
            n = torch.tensor([buf.size], dtype=torch.int64, device=dev)
            t = torch.from_numpy(buf).to(dev)
            hold += [n, t]
            reqs.append(self.dist.isend(n, peer, group=self.group))
            reqs.append(self.dist.isend(t, peer, group=self.group))
        for peer in recv_from:
            n = torch.zeros(1, dtype=torch.int64, device=dev)
            self.dist.recv(n, peer, group=self.group)
            t = torch.zeros(int(n.item()), dtype=torch.float64, device=dev)
            self.dist.recv(t, peer, group=self.group)
            out[peer] = t.cpu().numpy()
        for r in reqs:
            r.wait()
        return out

    def refresh_ghosts(self):
        """One exchange: the first owned site (with the bond right of it) goes left, the
        last owned site (with the bond left of it) goes right."""
        seg, eng = self.seg, self.engine
        r, R = seg.rank, seg.world
        sends, recv = {}, []
        if r > 0:
            s = seg.lo
            sends[r - 1] = pack(s, s + 1, eng.bond(s + 1), eng.site(s))
            recv.append(r - 1)
        if r < R - 1:
            s = seg.hi - 1
            sends[r + 1] = pack(s, s, eng.bond(s), eng.site(s))
            recv.append(r + 1)
        got = self._send_recv(sends, recv)
        for peer in recv:
            site, bond, lam, pairs, data = unpack(got[peer])
            dims = {c: len(v) for c, v in lam.items()}
            if bond == site:          # the bond left of the ghost site
                left, right = dims, eng.bond_dims(site + 1)
            else:                     # the bond right of it
                left, right = eng.bond_dims(site), dims
            eng.load(bond, lam, site, place_blocks(pairs, data, left, right))
        self.exchanges += 1

    def layer(self, sites, gate_of, f, chi, cutoff):
        """Apply one layer; returns the left sites this rank updated."""
        if self.seg.world > 1 and self.seg.straddles(sites):
            self.refresh_ghosts()
        mine = self.seg.updates(sites)
        self.engine.apply_layer(mine, [gate_of(s, f) for s in mine], chi, cutoff)
        return mine

    def gather(self, root: int = 0):
        """The owned sites and the bonds left of them, collected on `root` as
        ({bond: lambda dict}, {site: blocks}); other ranks get None."""
        seg, eng = self.seg, self.engine
        mine = [pack(s, s, eng.bond(s), eng.site(s)) for s in range(seg.lo, seg.hi)]
        if seg.rank != root:
            self._send_recv({root: np.concatenate([np.array([len(mine)], np.float64)] +
                                                  [np.concatenate([[b.size], b]) for b in mine])}, [])
            return None
        bonds, sites = {}, {}
        bufs = {seg.rank: mine}
        others = [r for r in range(seg.world) if r != root]
        got = self._send_recv({}, others)
        for r in others:
            flat, o, lst = got[r], 1, []
            for _ in range(int(flat[0])):
                n = int(flat[o])
                lst.append(flat[o + 1:o + 1 + n])
                o += 1 + n
            bufs[r] = lst
        for r in range(seg.world):
            for buf in bufs[r]:
                site, bond, lam, pairs, data = unpack(buf)
                bonds[bond] = lam
                sites[site] = (pairs, data)
        return bonds, sites
