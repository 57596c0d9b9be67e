"""Row-partitioned solve (Sec. 3.1, Eq. 4-5) through the C ABI: argument marshalling and
a communicator for the library's pc_comm callbacks.

Every step of the solve runs in the CUDA library (pc_dist_*). The library asks its
caller for two collectives, a sum of a few doubles over the ranks and a point-to-point
exchange of device buffers; `HostComm` provides both over a torch.distributed process
group that handles CPU tensors (gloo), staging each transfer through host memory. It is
the communicator the tests use, with several ranks sharing one GPU; a node with one GPU
per rank would pass a communicator that moves device buffers directly (NCCL), which this
repository does not contain.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch
import torch.distributed as dist

from . import pcloth as pc

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
P = ctypes.POINTER

ALLREDUCE_FN = ctypes.CFUNCTYPE(c_int32, c_void_p, c_void_p, c_int32, c_void_p)
EXCHANGE_FN = ctypes.CFUNCTYPE(c_int32, c_void_p, c_void_p, P(c_int64), P(c_int64), c_void_p, P(c_int64), P(c_int64),
                               c_void_p)


class pc_comm(ctypes.Structure):
    _fields_ = [("user", c_void_p), ("allreduce_sum", ALLREDUCE_FN), ("exchange", EXCHANGE_FN)]


def _declare(L):
    L.pc_dist_partition.argtypes = [c_int32, c_void_p, c_int32, c_void_p]
    L.pc_dist_halo.argtypes = [c_int32, c_void_p, c_int32, c_int64, c_void_p, c_void_p, P(c_int64), c_void_p]
    L.pc_dist_create.argtypes = [P(c_void_p), c_int32, c_int32, c_void_p, c_int64, c_int64]
    L.pc_dist_destroy.argtypes = [c_void_p]
    L.pc_dist_plan.argtypes = [c_void_p, P(pc.pc_bsr), P(pc_comm), c_void_p]
    L.pc_dist_sizes.argtypes = [c_void_p, P(c_int32), P(c_int32), P(c_int64), P(c_int64), P(c_int64), P(c_int64)]
    L.pc_dist_pcg_solve.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, P(pc.pc_solve_opts),
                                    P(pc_comm), P(pc.pc_solve_info), c_void_p]
    for name in ("pc_dist_partition", "pc_dist_halo", "pc_dist_create", "pc_dist_destroy", "pc_dist_plan",
                 "pc_dist_sizes", "pc_dist_pcg_solve"):
        getattr(L, name).restype = c_int32
    return L


_lib = _declare(pc.lib())


# --------------------------------------------------------------------------- host-only helpers


def partition(V: int, nranks: int, row_ptr: np.ndarray | None = None) -> np.ndarray:
    """Row blocks per rank (pc_dist_partition): int32[nranks + 1]."""
    out = np.zeros(nranks + 1, np.int32)
    rp = None if row_ptr is None else np.ascontiguousarray(row_ptr, np.int32)
    pc._check(_lib.pc_dist_partition(int(V), rp.ctypes.data_as(c_void_p) if rp is not None else None, int(nranks),
                                     out.ctypes.data_as(c_void_p)), "pc_dist_partition")
    return out


def halo(row_starts: np.ndarray, rank: int, remote: np.ndarray):
    """(sorted distinct halo columns, per-owner counts) of a rank (pc_dist_halo)."""
    rs = np.ascontiguousarray(row_starts, np.int32)
    rem = np.ascontiguousarray(remote, np.int32)
    out = np.zeros(max(len(rem), 1), np.int32)
    counts = np.zeros(len(rs) - 1, np.int64)
    n = c_int64()
    pc._check(_lib.pc_dist_halo(len(rs) - 1, rs.ctypes.data_as(c_void_p), int(rank), len(rem),
                                rem.ctypes.data_as(c_void_p), out.ctypes.data_as(c_void_p), ctypes.byref(n),
                                counts.ctypes.data_as(c_void_p)), "pc_dist_halo")
    return out[: n.value].copy(), counts


# --------------------------------------------------------------------------- communicator


class _DeviceBytes:
    """A CUDA byte range as an array-interface object (wrapped by torch without a copy)."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (int(nbytes),), "typestr": "|u1", "data": (int(ptr), False),
                                         "version": 3, "strides": None, "stream": None}


def _device_bytes(ptr: int, nbytes: int) -> torch.Tensor:
    return torch.as_tensor(_DeviceBytes(ptr, nbytes), device="cuda")


class HostComm:
    """pc_comm over a torch.distributed group that handles CPU tensors (gloo). Transfers go
    through host memory: the library's stream is synchronized, the bytes copied out,
    exchanged, and copied back before the callback returns."""

    def __init__(self, group=None):
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.calls = {"allreduce": 0, "exchange": 0}
        self._ar = ALLREDUCE_FN(self._allreduce_cb)
        self._ex = EXCHANGE_FN(self._exchange_cb)
        self.struct = pc_comm(None, self._ar, self._ex)
        self.error = None

    # -- tensor-level collectives (CPU tensors; the callbacks below stage device memory)
    def allreduce(self, t: torch.Tensor):
        """Sum over the ranks, added in rank order on every rank, so that every rank gets
        the same bits (the ranks take their stop decisions from these sums)."""
        parts = [torch.empty_like(t) for _ in range(self.world)]
        dist.all_gather(parts, t, group=self.group)
        acc = parts[0].clone()
        for p in parts[1:]:
            acc += p
        t.copy_(acc)

    def exchange(self, send: torch.Tensor, send_off, send_bytes, recv: torch.Tensor, recv_off, recv_bytes):
        """Byte exchange between CPU uint8 tensors: send[send_off[j]:+send_bytes[j]] goes
        to rank j, recv[recv_off[j]:+recv_bytes[j]] comes from rank j."""
        reqs = []
        for j in range(self.world):
            if j == self.rank:
                continue
            if recv_bytes[j] > 0:
                reqs.append(dist.irecv(recv[recv_off[j]: recv_off[j] + recv_bytes[j]], src=j, group=self.group))
            if send_bytes[j] > 0:
                reqs.append(dist.isend(send[send_off[j]: send_off[j] + send_bytes[j]].clone(), dst=j,
                                       group=self.group))
        for r in reqs:
            r.wait()

    # -- ctypes callbacks
    def _allreduce_cb(self, user, vals, n, stream):
        try:
            self.calls["allreduce"] += 1
            torch.cuda.ExternalStream(stream).synchronize() if stream else torch.cuda.synchronize()
            dev = _device_bytes(vals, 8 * n).view(torch.float64)
            host = dev.cpu()
            self.allreduce(host)
            dev.copy_(host)
            torch.cuda.current_stream().synchronize()
            return 0
        except Exception as e:  # reported by the library as PC_ERR_CUDA; kept for the caller
            self.error = e
            return 1

    def _exchange_cb(self, user, send, so, sb, recv, ro, rb, stream):
        try:
            self.calls["exchange"] += 1
            W = self.world
            so, sb, ro, rb = ([int(a[j]) for j in range(W)] for a in (so, sb, ro, rb))
            torch.cuda.ExternalStream(stream).synchronize() if stream else torch.cuda.synchronize()
            s_end = max([o + b for o, b in zip(so, sb)] + [0])
            r_end = max([o + b for o, b in zip(ro, rb)] + [0])
            hs = _device_bytes(send, s_end).cpu() if s_end > 0 else torch.zeros(0, dtype=torch.uint8)
            hr = torch.zeros(r_end, dtype=torch.uint8)
            self.exchange(hs, so, sb, hr, ro, rb)
            if r_end > 0:
                dr = _device_bytes(recv, r_end)
                for j in range(W):
                    if rb[j] > 0:
                        dr[ro[j]: ro[j] + rb[j]].copy_(hr[ro[j]: ro[j] + rb[j]])
                torch.cuda.current_stream().synchronize()
            return 0
        except Exception as e:
            self.error = e
            return 1


# --------------------------------------------------------------------------- the rank's solver


class DistSolver:
    """One rank of the row-partitioned solve: pc_dist_create / plan / pcg_solve."""

    def __init__(self, comm: HostComm, row_starts: np.ndarray, max_blocks: int, max_halo: int = 0):
        self.comm = comm
        self.row_starts = np.ascontiguousarray(row_starts, np.int32)
        self.rank = comm.rank
        self.row0 = int(self.row_starts[self.rank])
        self.row1 = int(self.row_starts[self.rank + 1])
        h = c_void_p()
        pc._check(_lib.pc_dist_create(ctypes.byref(h), self.rank, comm.world, self.row_starts.ctypes.data_as(c_void_p),
                                      int(max_blocks), int(max_halo)), "pc_dist_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) is not None:
            _lib.pc_dist_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, st, what):
        if st != pc.PC_OK and self.comm.error is not None:
            raise RuntimeError(f"{what}: communicator failed") from self.comm.error
        pc._check(st, what)

    def plan(self, row_ptr: torch.Tensor, col_idx: torch.Tensor, nnzb: int, stream=None):
        """row_ptr: the FULL system's device row pointers (this rank's slice is taken
        here by pointer offset); col_idx: the full column indices."""
        A = pc.pc_bsr()
        A.row_ptr = row_ptr.data_ptr() + 4 * self.row0
        A.col_idx = col_idx.data_ptr()
        A.cap = (col_idx.numel() // 4) * 4
        A.nnzb = int(nnzb)
        st = _lib.pc_dist_plan(self.handle, ctypes.byref(A), ctypes.byref(self.comm.struct), pc._stream(stream))
        self._raise(st, "pc_dist_plan")

    def sizes(self):
        r0, r1 = c_int32(), c_int32()
        nh, ns, no, nhb = c_int64(), c_int64(), c_int64(), c_int64()
        pc._check(_lib.pc_dist_sizes(self.handle, ctypes.byref(r0), ctypes.byref(r1), ctypes.byref(nh),
                                     ctypes.byref(ns), ctypes.byref(no), ctypes.byref(nhb)), "pc_dist_sizes")
        return {"row0": r0.value, "row1": r1.value, "n_halo": nh.value, "n_send": ns.value, "nnzb_own": no.value,
                "nnzb_halo": nhb.value}

    def solve(self, vals: torch.Tensor, dres_rows, b_rows: torch.Tensor, dv_rows: torch.Tensor, opts=None,
              stream=None, allow_not_converged=False):
        """vals: the full value array (indexed like col_idx); dres_rows, b_rows, dv_rows:
        this rank's rows (contiguous device tensors)."""
        info = pc.pc_solve_info()
        o = opts if opts is not None else pc.solve_opts()
        st = _lib.pc_dist_pcg_solve(self.handle, pc._ptr(vals), pc._ptr(dres_rows), pc._ptr(b_rows), pc._ptr(dv_rows),
                                    ctypes.byref(o), ctypes.byref(self.comm.struct), ctypes.byref(info),
                                    pc._stream(stream))
        if not (allow_not_converged and st == pc.PC_ERR_NOT_CONVERGED):
            self._raise(st, "pc_dist_pcg_solve")
        return info, st
