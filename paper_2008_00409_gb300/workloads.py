"""Seeded synthetic cloth workloads: meshes, pins, initial state, per-step contact pairs.

This module produces inputs only. It holds none of the integrator's arithmetic (no
forces, Jacobians, masses or solver steps): both the CUDA path and the FP64 oracle
consume exactly what it returns, cast to their own types.

The paper (Sec. 5) measures on garment datasets that are not available here; these
regular and jittered grids stand in for them at the same sizes (0.5-1.65M triangles,
multi-layer pieces, contact pairs that change every step, Sec. 3 and Sec. 5).

Randomness is counter-based: every draw is the SplitMix64 output (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) at an explicit
position of a sequence keyed by ``(seed, stream)``, so a workload is identical on any
machine and any numpy version, and a step's contacts depend only on ``(seed, step)``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each 64-bit counter value (vectorised, wraps mod 2**64)."""
    with np.errstate(over="ignore"):
        z = counter.astype(np.uint64) * np.uint64(1) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _stream_base(seed: int, stream: int) -> np.uint64:
    """Starting state of the (seed, stream) sequence: one SplitMix64 mix of both ids."""
    key = np.array([((seed & 0xFFFFFFFFFFFF) << 16) ^ (stream & 0xFFFF)], dtype=np.uint64)
    return splitmix64(key)[0]


def _counters_at(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        return _stream_base(seed, stream) + np.asarray(index, dtype=np.uint64) * _GOLDEN


def uniform_at(seed: int, stream: int, index) -> np.ndarray:
    """Uniform float64 draws in [0, 1) at explicit positions of the (seed, stream) sequence."""
    bits = splitmix64(_counters_at(seed, stream, index)) >> np.uint64(11)
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniform float64 draws in [0, 1): positions offset .. offset+n-1 of the sequence."""
    return uniform_at(seed, stream, np.arange(offset, offset + n, dtype=np.uint64))


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal draws (Box-Muller on two uniform streams)."""
    u1 = uniform(seed, stream, n)
    u2 = uniform(seed, stream + 1, n)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def randint_at(seed: int, stream: int, index, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive) at explicit sequence positions."""
    u = uniform_at(seed, stream, index)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


def randint(seed: int, stream: int, n: int, lo: int, hi: int, offset: int = 0) -> np.ndarray:
    """n integers uniform in [lo, hi] (inclusive)."""
    return randint_at(seed, stream, np.arange(offset, offset + n, dtype=np.uint64), lo, hi)


# --------------------------------------------------------------------------- material


@dataclasses.dataclass(frozen=True)
class Material:
    """Cloth material: the values every workload uses unless it says otherwise."""

    rho: float = 0.1          # area density, kg/m^2
    young: float = 5e3        # membrane Young's modulus x thickness, N/m
    poisson: float = 0.3
    k_bend: float = 1e-4      # dihedral bending stiffness, N*m
    k_contact: float = 1e3    # contact penalty stiffness, N/m
    gravity: tuple = (0.0, 0.0, -9.81)
    damp_mass: float = 0.0    # Rayleigh damping alpha (1/s): f_d = -(alpha M + beta K) v
    damp_stiff: float = 0.0   # Rayleigh damping beta (s)
    contact_thickness: float = 0.0  # m: 0 = hold penalty, > 0 = one-sided thickness penalty

    def as_array(self) -> np.ndarray:
        return np.array([self.rho, self.young, self.poisson, self.k_bend, self.k_contact,
                         *self.gravity, self.damp_mass, self.damp_stiff, self.contact_thickness],
                        dtype=np.float64)


# --------------------------------------------------------------------------- meshes


@dataclasses.dataclass
class Sheet:
    """One rectangular grid piece inside a workload (for contact sampling)."""

    nx: int
    ny: int
    vbase: int            # first vertex index of the piece
    tbase: int            # first triangle index of the piece
    flip: np.ndarray      # bool [ny-1, nx-1]: quad uses the (i+1,j)-(i,j+1) diagonal


@dataclasses.dataclass
class Workload:
    name: str
    rest: np.ndarray          # float32 [V, 3] rest positions (planar per piece)
    tris: np.ndarray          # int32 [T, 3], counter-clockwise seen from +z
    pins: np.ndarray          # int32 [n_pins]
    x0: np.ndarray            # float32 [V, 3] initial positions
    v0: np.ndarray            # float32 [V, 3] initial velocities
    h: float
    material: Material
    sheets: list
    seed: int
    contact_kind: str = "none"    # none | grid | interlayer | batch | proximity
    contact_frac: float = 0.0     # pairs per vertex (proximity: the capacity per vertex)
    contact_radius: int = 8
    steps: int = 1
    parts: list = None            # batch: the garments, in row order
    inst_rows: np.ndarray = None  # batch: first row of each garment, then V

    @property
    def V(self) -> int:
        return int(self.rest.shape[0])

    @property
    def T(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_contacts(self) -> int:
        if self.contact_kind == "batch":
            return int(sum(p.n_contacts for p in self.parts))
        return int(round(self.contact_frac * self.V)) if self.contact_kind != "none" else 0

    def contacts(self, step: int):
        """Contact pairs for one step: (pairs int32 [P,4] = (p,a,b,c), w float32 [P,3])."""
        if self.contact_kind == "none" or self.n_contacts == 0:
            return np.zeros((0, 4), np.int32), np.zeros((0, 3), np.float32)
        if self.contact_kind == "grid":
            return grid_contacts(self, step)
        if self.contact_kind == "interlayer":
            return interlayer_contacts(self, step)
        if self.contact_kind == "proximity":
            raise ValueError("proximity contacts come from the query at the current positions")
        if self.contact_kind == "batch":
            ps, ws = [], []
            for part, vb in zip(self.parts, self.inst_rows[:-1]):
                p, w = part.contacts(step)
                ps.append(p + np.int32(vb))
                ws.append(w)
            return np.concatenate(ps).astype(np.int32), np.concatenate(ws).astype(np.float32)
        raise ValueError(self.contact_kind)


def _quad_tris(nx: int, ny: int, flip: np.ndarray) -> np.ndarray:
    """Two counter-clockwise triangles per quad; quad (i, j) emits triangles 2q and 2q+1."""
    j, i = np.meshgrid(np.arange(ny - 1), np.arange(nx - 1), indexing="ij")
    v00 = j * nx + i
    v10 = v00 + 1
    v01 = v00 + nx
    v11 = v01 + 1
    f = flip.astype(bool)
    t0 = np.where(f[..., None], np.stack([v00, v10, v01], -1), np.stack([v00, v10, v11], -1))
    t1 = np.where(f[..., None], np.stack([v10, v11, v01], -1), np.stack([v00, v11, v01], -1))
    return np.stack([t0, t1], axis=2).reshape(-1, 3).astype(np.int32)


def quad_triangle(nx: int, flip: np.ndarray, i: np.ndarray, j: np.ndarray, upper: np.ndarray) -> np.ndarray:
    """Vertex triple of triangle `upper` (0/1) of quads (i, j), matching _quad_tris."""
    v00 = j * nx + i
    v10 = v00 + 1
    v01 = v00 + nx
    v11 = v01 + 1
    f = flip[j, i].astype(bool)
    up = upper.astype(bool)
    a0 = np.stack([v00, v10, np.where(f, v01, v11)], -1)
    a1 = np.stack([np.where(f, v10, v00), v11, v01], -1)
    return np.where(up[:, None], a1, a0)


def grid_piece(nx: int, ny: int, width: float, height: float, *, z: float = 0.0,
               jitter: float = 0.0, flip_prob: float = 0.0, seed: int = 0, stream: int = 0):
    """Rest positions and triangles of one nx x ny grid piece.

    `jitter` moves interior vertices in-plane by a uniform offset in
    [-jitter, jitter] x grid spacing; `flip_prob` flips each quad's diagonal.
    """
    dx = width / (nx - 1)
    dy = height / (ny - 1)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    px = ii * dx
    py = jj * dy
    if jitter > 0.0:
        n = nx * ny
        ox = (2.0 * uniform(seed, stream + 10, n) - 1.0).reshape(ny, nx) * jitter * dx
        oy = (2.0 * uniform(seed, stream + 11, n) - 1.0).reshape(ny, nx) * jitter * dy
        interior = (ii > 0) & (ii < nx - 1) & (jj > 0) & (jj < ny - 1)
        px = px + np.where(interior, ox, 0.0)
        py = py + np.where(interior, oy, 0.0)
    rest = np.stack([px, py, np.full_like(px, z)], -1).reshape(-1, 3)
    if flip_prob > 0.0:
        flip = (uniform(seed, stream + 12, (nx - 1) * (ny - 1)) < flip_prob).reshape(ny - 1, nx - 1)
    else:
        flip = np.zeros((ny - 1, nx - 1), bool)
    return rest.astype(np.float32), _quad_tris(nx, ny, flip), flip


def _assemble_pieces(pieces):
    rests, tris, sheets = [], [], []
    vb = tb = 0
    for (nx, ny, rest, tri, flip) in pieces:
        rests.append(rest)
        tris.append(tri + vb)
        sheets.append(Sheet(nx, ny, vb, tb, flip))
        vb += rest.shape[0]
        tb += tri.shape[0]
    return np.concatenate(rests), np.concatenate(tris).astype(np.int32), sheets


def _corner_pins(sheets) -> np.ndarray:
    """Two corners of each piece's top edge (j = ny - 1)."""
    pins = []
    for s in sheets:
        pins += [s.vbase + (s.ny - 1) * s.nx, s.vbase + (s.ny - 1) * s.nx + s.nx - 1]
    return np.array(pins, np.int32)


def square_cloth(n: int, *, seed: int, z_jitter: float = 1e-4, size: float = 1.0,
                 contact_frac: float = 0.0, name: str | None = None, steps: int = 20) -> Workload:
    """n x n vertex square cloth (diagonal triangulation), two top corners pinned.

    Initial positions get a seeded N(0, z_jitter) offset in z; rest stays flat.
    """
    rest, tri, flip = grid_piece(n, n, size, size)
    rest, tris, sheets = _assemble_pieces([(n, n, rest, tri, flip)])
    x0 = rest.astype(np.float64).copy()
    if z_jitter > 0.0:
        x0[:, 2] += z_jitter * normal(seed, 1, rest.shape[0])
    return Workload(name or f"square{n}", rest, tris, _corner_pins(sheets), x0.astype(np.float32),
                    np.zeros_like(rest), 1.0 / 200.0, Material(), sheets, seed,
                    contact_kind="grid" if contact_frac > 0 else "none", contact_frac=contact_frac,
                    steps=steps)


def training_cloth(n: int, *, seed: int, contact_frac: float = 0.02, steps: int = 250) -> Workload:
    """n x n square cloth with 1 to 4 pins drawn on its boundary and grid contacts: the
    trajectories that train the learned warm start."""
    wl = square_cloth(n, seed=seed, contact_frac=contact_frac, steps=steps, name=f"train{n}-{seed}")
    ring = np.concatenate([np.arange(n), (n - 1) * n + np.arange(n), n * np.arange(1, n - 1),
                           n * np.arange(1, n - 1) + n - 1])  # bottom, top, left, right edges
    k = int(randint(seed, 600, 1, 1, 4)[0])
    keys = splitmix64(_counters_at(seed, 601, np.arange(ring.size, dtype=np.uint64)))
    wl.pins = np.sort(ring[np.argsort(keys, kind="stable")[:k]]).astype(np.int32)
    return wl


def stacked_sheets(n: int = 526, layers: int = 3, *, seed: int, gap: float = 5e-4, size: float = 1.0,
                   jitter: float = 0.2, flip_prob: float = 0.1, contact_frac: float = 0.05,
                   steps: int = 10, name: str | None = None) -> Workload:
    """`layers` jittered n x n sheets stacked `gap` apart with random edge flips."""
    pieces = []
    for s in range(layers):
        rest, tri, flip = grid_piece(n, n, size, size, z=s * gap, jitter=jitter, flip_prob=flip_prob,
                                     seed=seed, stream=100 * (s + 1))
        pieces.append((n, n, rest, tri, flip))
    rest, tris, sheets = _assemble_pieces(pieces)
    return Workload(name or f"stack{layers}x{n}", rest, tris, _corner_pins(sheets), rest.copy(),
                    np.zeros_like(rest), 1.0 / 200.0, Material(), sheets, seed,
                    contact_kind="interlayer" if contact_frac > 0 else "none",
                    contact_frac=contact_frac, steps=steps)


def garment(n: int, *, seed: int, stream: int, contact_frac: float = 0.01, jitter: float = 0.2) -> Workload:
    """One jittered n x n piece standing in for a garment of the batched workload."""
    rest, tri, flip = grid_piece(n, n, 1.0, 1.0, jitter=jitter, flip_prob=0.1, seed=seed, stream=stream)
    rest, tris, sheets = _assemble_pieces([(n, n, rest, tri, flip)])
    x0 = rest.astype(np.float64).copy()
    x0[:, 2] += 1e-4 * normal(seed, stream + 7, rest.shape[0])
    return Workload(f"garment{n}", rest, tris, _corner_pins(sheets), x0.astype(np.float32),
                    np.zeros_like(rest), 1.0 / 200.0, Material(), sheets, seed + stream,
                    contact_kind="grid" if contact_frac > 0 else "none", contact_frac=contact_frac)


def garment_batch(count: int = 64, *, seed: int, tmin: float = 2e3, tmax: float = 2e5):
    """`count` garments with triangle counts drawn log-uniform in [tmin, tmax]."""
    u = uniform(seed, 500, count)
    tcount = np.exp(np.log(tmin) + u * (np.log(tmax) - np.log(tmin)))
    sides = np.round(np.sqrt(tcount / 2.0)).astype(int) + 1
    return [garment(int(s), seed=seed, stream=1000 + 16 * k) for k, s in enumerate(sides)]


def batch_union(parts, name: str = "batch") -> Workload:
    """Disjoint union of workloads, stacked in row order (one block-diagonal system).

    Vertex indices of part k are shifted by inst_rows[k]; contacts are each part's own,
    shifted the same way, so no element couples two parts.
    """
    offs = np.cumsum([0] + [p.V for p in parts])
    toffs = np.cumsum([0] + [p.T for p in parts])
    rest = np.concatenate([p.rest for p in parts])
    tris = np.concatenate([p.tris + np.int32(o) for p, o in zip(parts, offs[:-1])]).astype(np.int32)
    pins = np.concatenate([p.pins + np.int32(o) for p, o in zip(parts, offs[:-1])]).astype(np.int32)
    sheets = []
    for p, vo, to in zip(parts, offs[:-1], toffs[:-1]):
        for s in p.sheets:
            sheets.append(Sheet(s.nx, s.ny, s.vbase + int(vo), s.tbase + int(to), s.flip))
    return Workload(name, rest, tris, pins, np.concatenate([p.x0 for p in parts]),
                    np.concatenate([p.v0 for p in parts]), parts[0].h, parts[0].material, sheets, parts[0].seed,
                    contact_kind="batch", steps=parts[0].steps, parts=list(parts),
                    inst_rows=offs.astype(np.int32))


def garment_batch_union(count: int = 64, *, seed: int = 20080409 + 4, tmin: float = 2e3, tmax: float = 2e5):
    """The batched workload: `count` log-uniform garments as one union (block diagonal)."""
    return batch_union(garment_batch(count, seed=seed, tmin=tmin, tmax=tmax), name=f"batch{count}")


# --------------------------------------------------------------------------- contacts


def _pick_vertices(wl: Workload, step: int, count: int, stream: int) -> np.ndarray:
    """`count` distinct vertices, chosen by ranking counter-based keys."""
    keys = splitmix64(_counters_at(wl.seed, stream, np.arange(wl.V, dtype=np.uint64) + np.uint64(step * wl.V)))
    return np.sort(np.argsort(keys, kind="stable")[:count]).astype(np.int64)


def _dirichlet3(seed: int, stream: int, n: int, offset: int) -> np.ndarray:
    e = -np.log1p(-uniform(seed, stream, 3 * n, offset)).reshape(n, 3)
    e = np.maximum(e, 1e-12)
    w = e / e.sum(1, keepdims=True)
    return w.astype(np.float32)


def grid_contacts(wl: Workload, step: int):
    """Pair round(frac * V) vertices with random triangles within `radius` grid cells.

    Each chosen vertex p at grid cell (i, j) draws a quad offset (di, dj) in
    [-radius, radius]^2 and one of the quad's two triangles; a draw that leaves the
    piece or whose triangle contains p is redrawn (up to 64 rounds, then the nearest
    non-incident triangle in scan order is taken). Weights are Dirichlet(1, 1, 1).
    """
    P = wl.n_contacts
    verts = _pick_vertices(wl, step, P, stream=2000)
    pairs = np.zeros((P, 4), np.int64)
    r = wl.contact_radius
    # locate each vertex in its sheet
    sheet_of = np.zeros(P, np.int64)
    for s_idx, s in enumerate(wl.sheets):
        m = (verts >= s.vbase) & (verts < s.vbase + s.nx * s.ny)
        sheet_of[m] = s_idx
    pending = np.arange(P)
    for attempt in range(64):
        if pending.size == 0:
            break
        n = pending.size
        idx_draw = (step * 64 + attempt) * wl.V + pending
        di = randint_at(wl.seed, 3000, idx_draw, -r, r)
        dj = randint_at(wl.seed, 3001, idx_draw, -r, r)
        up = randint_at(wl.seed, 3002, idx_draw, 0, 1)
        keep = np.zeros(n, bool)
        for s_idx, s in enumerate(wl.sheets):
            m = sheet_of[pending] == s_idx
            if not m.any():
                continue
            local = verts[pending[m]] - s.vbase
            pi, pj = local % s.nx, local // s.nx
            qi, qj = pi + di[m], pj + dj[m]
            ok = (qi >= 0) & (qi < s.nx - 1) & (qj >= 0) & (qj < s.ny - 1)
            qi_c = np.clip(qi, 0, s.nx - 2)
            qj_c = np.clip(qj, 0, s.ny - 2)
            tri = quad_triangle(s.nx, s.flip, qi_c, qj_c, up[m]) + s.vbase
            ok &= ~(tri == verts[pending[m]][:, None]).any(1)
            idx = pending[m][ok]
            pairs[idx, 0] = verts[idx]
            pairs[idx, 1:] = tri[ok]
            sub = np.zeros(n, bool)
            sub[np.nonzero(m)[0][ok]] = True
            keep |= sub
        pending = pending[~keep]
    for k in pending:  # deterministic fallback: first non-incident triangle of the next quad row
        s = wl.sheets[sheet_of[k]]
        local = verts[k] - s.vbase
        pi, pj = local % s.nx, local // s.nx
        qj = pj + 1 if pj + 1 < s.ny - 1 else pj - 2
        qi = min(max(pi, 0), s.nx - 2)
        tri = quad_triangle(s.nx, s.flip, np.array([qi]), np.array([qj]), np.array([0]))[0] + s.vbase
        pairs[k] = (verts[k], *tri)
    w = _dirichlet3(wl.seed, 3003, P, offset=step * wl.V * 3)
    return pairs.astype(np.int32), w


def interlayer_contacts(wl: Workload, step: int):
    """Pair round(frac * V) vertices with a triangle of an adjacent sheet at the same (i, j).

    The partner triangle lies in a quad touching grid position (i, j) of the
    neighbouring layer (upper or lower, drawn at random where both exist).
    """
    P = wl.n_contacts
    verts = _pick_vertices(wl, step, P, stream=4000)
    L = len(wl.sheets)
    pairs = np.zeros((P, 4), np.int64)
    off = step * wl.V
    ud = randint(wl.seed, 4001, P, 0, 1, offset=off)
    qsel_i = randint(wl.seed, 4002, P, 0, 1, offset=off)
    qsel_j = randint(wl.seed, 4003, P, 0, 1, offset=off)
    up = randint(wl.seed, 4004, P, 0, 1, offset=off)
    sizes = np.array([s.nx * s.ny for s in wl.sheets])
    bases = np.array([s.vbase for s in wl.sheets])
    layer = np.searchsorted(bases, verts, side="right") - 1
    for l in range(L):
        m = layer == l
        if not m.any():
            continue
        s = wl.sheets[l]
        if L == 1:
            raise ValueError("interlayer contacts need at least two sheets")
        partner = np.where(ud[m] == 1, l + 1, l - 1)
        partner = np.where(partner < 0, l + 1, partner)
        partner = np.where(partner >= L, l - 1, partner)
        local = verts[m] - s.vbase
        pi, pj = local % s.nx, local // s.nx
        for pl in np.unique(partner):
            mm = partner == pl
            t = wl.sheets[pl]
            qi = np.clip(pi[mm] - qsel_i[m][mm], 0, t.nx - 2)
            qj = np.clip(pj[mm] - qsel_j[m][mm], 0, t.ny - 2)
            tri = quad_triangle(t.nx, t.flip, qi, qj, up[m][mm]) + t.vbase
            idx = np.nonzero(m)[0][mm]
            pairs[idx, 0] = verts[idx]
            pairs[idx, 1:] = tri
    del sizes
    w = _dirichlet3(wl.seed, 4005, P, offset=step * wl.V * 3)
    return pairs.astype(np.int32), w


# --------------------------------------------------------------------------- named workloads

SEED_BASE = 20080409


def small_square() -> Workload:
    """64 x 64 cloth, 1 m x 1 m, two corners pinned, no contacts, 20 steps."""
    return square_cloth(64, seed=SEED_BASE + 1, steps=20, name="square64")


def dynamic_square(n: int = 512) -> Workload:
    """512 x 512 cloth, 2% of vertices in contact pairs regenerated every step."""
    return square_cloth(n, seed=SEED_BASE + 2, contact_frac=0.02, steps=20, name=f"square{n}-contacts")


def paper_scale(n: int = 526, layers: int = 3) -> Workload:
    """Three stacked 526 x 526 sheets (about 1.65M triangles), 5% inter-layer contacts."""
    return stacked_sheets(n, layers, seed=SEED_BASE + 3, steps=10, name=f"stack{layers}x{n}")


def warm_start_eval(n: int = 708) -> Workload:
    """708 x 708 cloth (about 1M triangles), 2% contacts: the learned warm start's test cloth."""
    return square_cloth(n, seed=SEED_BASE + 5, contact_frac=0.02, steps=10, name=f"square{n}-contacts")


def warm_start_training(n: int = 256, count: int = 8, steps: int = 250):
    """`count` n x n cloths with random boundary pins and 2% contacts, `steps` steps each
    (8 x 250 = 2,000 integrator steps on 256 x 256 cloths by default)."""
    return [training_cloth(n, seed=SEED_BASE + 5 + 1000 * (k + 1), steps=steps) for k in range(count)]


def proximity_stack(n: int = 526, layers: int = 3, *, delta: float = 5.5e-4, per_vertex: float = 6.0,
                    seed: int = SEED_BASE + 3, steps: int = 10, name: str | None = None) -> Workload:
    """The stacked sheets (0.5 mm apart) with the one-sided thickness contact model: the
    contacts of each step are the vertex-triangle pairs closer than `delta` at the
    step's positions (found by the proximity query), room for `per_vertex` pairs per
    vertex."""
    wl = stacked_sheets(n, layers, seed=seed, contact_frac=0.0, steps=steps,
                        name=name or f"stack{layers}x{n}-proximity")
    wl.material = dataclasses.replace(wl.material, contact_thickness=delta)
    wl.contact_kind = "proximity"
    wl.contact_frac = per_vertex
    return wl


WORKLOADS = {
    "square64": small_square,
    "square512-contacts": dynamic_square,
    "stack3x526": paper_scale,
    "stack3x526-proximity": proximity_stack,
}
