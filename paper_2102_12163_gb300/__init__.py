"""GB300 implementation of the multiresolution-adaptive lattice Boltzmann step
(Bellotti, Gouarin, Graille, Massot, arXiv 2102.12163).

The computation lives in the CUDA library ``libmrlbm.so`` behind the C ABI of
``include/mrlbm.h``; this package marshals arguments to it (``capi``) and uses
PyTorch only for the device workspace and the CUDA stream.  ``workloads``
describes the seeded test problems.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import capi, workloads
from .capi import MR_FP32_MIXED, MR_FP64, MRError

__all__ = ["MRLBM", "MRError", "capi", "workloads", "MR_FP64", "MR_FP32_MIXED"]

_EQ = {workloads.EQ_ADVECTION: capi.MR_EQ_ADVECTION, workloads.EQ_BURGERS: capi.MR_EQ_BURGERS,
       workloads.EQ_SW: capi.MR_EQ_SW_VEC, workloads.EQ_EULER: capi.MR_EQ_EULER_VEC,
       workloads.EQ_SW_D1Q3: capi.MR_EQ_SW_D1Q3, workloads.EQ_SW_D1Q5: capi.MR_EQ_SW_D1Q5}


def _desc(inst: "workloads.Instance") -> capi.mr_instance_desc:
    d = capi.mr_instance_desc()
    d.Jmin, d.Jmax, d.gamma, d.mu_bar, d.bc, d.eq = inst.Jmin, inst.Jmax, inst.gamma, inst.mu_bar, inst.bc, _EQ[inst.eq]
    d.eps, d.a, d.b, d.lambda_ = inst.eps, inst.a, inst.b, inst.lam
    s = list(inst.s) + [1.0] * 3
    for j in range(3):
        d.s[j] = s[j]
    d.eq_param = inst.eqp
    d.collision = inst.collision
    return d


def probe_latency(device: str = "cuda:0") -> dict:
    """SM cycles of one warp-to-warp hand-over through global memory, through
    shared memory, of a bare block barrier, and through a global line the
    block has not touched before (mr_probe_latency)."""
    import torch

    lib = capi.load()
    dev = torch.device(device)
    nbytes = 4096 + 4096 * 128
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    out = (ctypes.c_double * 4)()
    capi.check(None, lib.mr_probe_latency(ctypes.c_void_p(scratch.data_ptr()), nbytes,
                                          ctypes.c_void_p(stream.cuda_stream), out))
    return {"global_handover_cycles": out[0], "shared_handover_cycles": out[1], "barrier_cycles": out[2],
            "fresh_line_handover_cycles": out[3]}


class MRLBM:
    """One context of the C ABI holding one or many instances on one GPU.

    A single instance is created through ``mr_mesh_init`` + ``lbm_scheme`` (the
    paper's problem statement); several through ``mr_batch_create``.
    """

    def __init__(self, instances, precision: int = MR_FP64, device: str = "cuda:0", block: int | None = None,
                 stream=None):
        import torch

        self.lib = capi.load()
        self.instances = list(instances) if isinstance(instances, (list, tuple)) else [instances]
        self.precision = precision
        self.device = torch.device(device)
        h = ctypes.c_void_p()
        if len(self.instances) == 1:
            inst = self.instances[0]
            capi.check(None, self.lib.mr_mesh_init(ctypes.byref(h), inst.Jmin, inst.Jmax, inst.gamma, inst.eps,
                                                   inst.a, inst.b, inst.bc, inst.mu_bar, precision))
            self.h = h
            s = (ctypes.c_double * 3)(*(list(inst.s) + [1.0] * 3)[:3])
            eqp = ctypes.c_double(inst.eqp)
            capi.check(self.h, self.lib.lbm_scheme(self.h, 1, inst.q, inst.lam, s, _EQ[inst.eq], ctypes.byref(eqp)))
            if inst.collision:
                capi.check(self.h, self.lib.mr_set_collision(self.h, inst.collision))
        else:
            arr = (capi.mr_instance_desc * len(self.instances))(*[_desc(i) for i in self.instances])
            capi.check(None, self.lib.mr_batch_create(ctypes.byref(h), arr, len(self.instances), precision))
            self.h = h
        nbytes = ctypes.c_size_t()
        capi.check(self.h, self.lib.mr_workspace_size(self.h, ctypes.byref(nbytes)))
        self.workspace_bytes = nbytes.value
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            # caller-owned workspace (torch allocations are 512-byte aligned)
            self.ws = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
        if block is not None:
            self.set_launch(block, 0)
        capi.check(self.h, self.lib.mr_bind(self.h, ctypes.c_void_p(self.ws.data_ptr()), self.workspace_bytes,
                                            ctypes.c_void_p(self.stream.cuda_stream)))

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.lib.mr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_launch(self, block: int, grid: int = 0):
        """Threads per block (128, 256, 512 or 1024) and blocks (0: one resident wave)."""
        capi.check(self.h, self.lib.mr_set_launch(self.h, block, grid))

    def set_order(self, by_fields: bool):
        """Work-queue order: field count first (default) or size alone."""
        capi.check(self.h, self.lib.mr_set_order(self.h, 1 if by_fields else 0))

    def autotune(self, nsteps: int = 8) -> dict:
        """Time nsteps steps under every block size (with the current queue
        order) and keep the fastest; the state is restored, so results are
        unchanged."""
        import torch

        scratch = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
        b, o, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        capi.check(self.h, self.lib.mr_autotune(self.h, nsteps, ctypes.c_void_p(scratch.data_ptr()),
                                                self.workspace_bytes, ctypes.byref(b), ctypes.byref(o),
                                                ctypes.byref(ms)))
        del scratch
        return {"block": b.value, "order_by_fields": bool(o.value), "ms_per_trial": ms.value, "steps": nsteps}

    def capture(self, nsteps: int):
        """A CUDA graph holding the persistent launches of nsteps adaptive steps
        (one per kernel variant the batch needs, forked from and joined back to
        this context's stream); ``replay()`` advances every instance by nsteps."""
        import torch

        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            capi.check(self.h, self.lib.mr_advance(self.h, nsteps))
        return g

    # -- state -------------------------------------------------------------
    def initial_data(self) -> np.ndarray:
        return np.concatenate([np.ascontiguousarray(i.m0, dtype=np.float64).ravel() for i in self.instances])

    def set_initial(self, m_cons=None):
        """Initial conserved moments: numpy (host) or torch tensor (host or device)."""
        if m_cons is None:
            m_cons = self.initial_data()
        if isinstance(m_cons, np.ndarray):
            m_cons = np.ascontiguousarray(m_cons, dtype=np.float64)
            ptr, n = m_cons.ctypes.data, m_cons.size
        else:
            ptr, n = m_cons.data_ptr(), m_cons.numel()
        capi.check(self.h, self.lib.mr_set_initial(self.h, ctypes.c_void_p(ptr), n))
        self._keep = m_cons

    def set_state(self, inst: int, R: np.ndarray, values: np.ndarray):
        import torch

        Rt = torch.as_tensor(np.ascontiguousarray(R, dtype=np.uint8)).to(self.device)
        Vt = torch.as_tensor(np.ascontiguousarray(values, dtype=np.float64)).to(self.device)
        torch.cuda.current_stream(self.device).synchronize()
        capi.check(self.h, self.lib.mr_set_state(self.h, inst, ctypes.c_void_p(Rt.data_ptr()),
                                                 ctypes.c_void_p(Vt.data_ptr())))
        self.sync()

    # -- stepping ----------------------------------------------------------
    def adapt(self):
        capi.check(self.h, self.lib.mr_adapt(self.h))

    def lbm_step(self):
        capi.check(self.h, self.lib.lbm_step(self.h))

    def advance(self, nsteps: int):
        capi.check(self.h, self.lib.mr_advance(self.h, nsteps))

    def sync(self):
        capi.check(self.h, self.lib.mr_sync(self.h))

    # -- results -----------------------------------------------------------
    def leaves(self, inst: int = 0):
        n = ctypes.c_long()
        capi.check(self.h, self.lib.mr_get_leaves(self.h, inst, None, None, None, 0, ctypes.byref(n)))
        cap = max(n.value, 1)
        q = self.instances[inst].q
        lv = np.zeros(cap, np.int32)
        ix = np.zeros(cap, np.int64)
        f = np.zeros((q, cap), np.float64)
        capi.check(self.h, self.lib.mr_get_leaves(
            self.h, inst, lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
            ix.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            cap, ctypes.byref(n)))
        k = n.value
        return lv[:k], ix[:k], f[:, :k]

    def moments(self, inst: int = 0):
        n = ctypes.c_long()
        capi.check(self.h, self.lib.mr_get_moments(self.h, inst, None, 0, ctypes.byref(n)))
        cap = max(n.value, 1)
        m = np.zeros((self.instances[inst].nf, cap), np.float64)
        capi.check(self.h, self.lib.mr_get_moments(self.h, inst, m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                   cap, ctypes.byref(n)))
        return m[:, :n.value]

    def finest(self, inst: int = 0) -> np.ndarray:
        ins = self.instances[inst]
        out = np.zeros((ins.nf, 1 << ins.Jmax), np.float64)
        capi.check(self.h, self.lib.mr_get_finest(self.h, inst, ctypes.c_void_p(out.ctypes.data)))
        return out

    def tree(self, inst: int = 0) -> np.ndarray:
        ins = self.instances[inst]
        S = (1 << (ins.Jmax + 1)) - (1 << ins.Jmin)
        R = np.zeros(S, np.uint8)
        capi.check(self.h, self.lib.mr_get_tree(self.h, inst, ctypes.c_void_p(R.ctypes.data)))
        return R

    def audit(self, inst: int = 0):
        ins = self.instances[inst]
        m = np.zeros(3, np.float64)
        r = ctypes.c_double()
        capi.check(self.h, self.lib.mr_audit(self.h, inst, m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             ctypes.byref(r)))
        return m[:ins.nf], r.value

    def summary(self, mass_out=None, nleaf_out=None):
        """Per-instance FP64 conserved totals (n, 3) and leaf counts (n,) in one
        device-to-host copy each; pass preallocated (pinned) outputs to reuse them."""
        n = len(self.instances)
        m = mass_out if mass_out is not None else np.zeros((n, 3), np.float64)
        c = nleaf_out if nleaf_out is not None else np.zeros(n, np.int32)
        mp = m.data_ptr() if hasattr(m, "data_ptr") else m.ctypes.data
        cp = c.data_ptr() if hasattr(c, "data_ptr") else c.ctypes.data
        capi.check(self.h, self.lib.mr_get_summary(self.h, ctypes.cast(mp, ctypes.POINTER(ctypes.c_double)),
                                                   ctypes.cast(cp, ctypes.POINTER(ctypes.c_int))))
        return m, c

    def near_ties(self, inst: int = 0) -> int:
        """Threshold and Harten decisions of instance inst within 1e-12 relative
        of their threshold since its initial state."""
        n = ctypes.c_longlong()
        capi.check(self.h, self.lib.mr_near_ties(self.h, inst, ctypes.byref(n)))
        return n.value

    def step_passes(self, inst: int = 0):
        """(steps, team barriers) of instance inst since its initial state."""
        st, ps = ctypes.c_ulonglong(), ctypes.c_ulonglong()
        capi.check(self.h, self.lib.mr_step_passes(self.h, inst, ctypes.byref(st), ctypes.byref(ps)))
        return st.value, ps.value

    def stats(self):
        u, s, lv = ctypes.c_ulonglong(), ctypes.c_ulonglong(), ctypes.c_longlong()
        capi.check(self.h, self.lib.mr_stats(self.h, ctypes.byref(u), ctypes.byref(s), ctypes.byref(lv)))
        return u.value, s.value, lv.value

    def phase_times(self, inst: int = 0):
        """SM cycles per phase of instance inst (phase-timer build only)."""
        arr = (ctypes.c_ulonglong * 16)()
        rc = self.lib.mr_phase_times(self.h, inst, arr, 16)
        if rc not in (capi.MR_OK, capi.MR_ERR_STATE):
            capi.check(self.h, rc)
        return dict(zip(capi.PHASES, arr[: len(capi.PHASES)]))

    def launches(self) -> int:
        n, l = ctypes.c_int(), ctypes.c_longlong()
        capi.check(self.h, self.lib.mr_info(self.h, ctypes.byref(n), ctypes.byref(l)))
        return l.value
