"""Python binding of the RVEA library: torch owns the device memory and the
streams, the CUDA library does every step of every generation.

    run = Run(m=3, d=5000, N=9870, H=139, problem=DTLZ1_LINEAR, t_max=1000)
    run.step(1000)
    F, valid = run.objectives()
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np
import torch

from ._native import (DTLZ1_LINEAR, DTLZ2_SPHERE, DTLZ3_SPHERE, DTLZ4_SPHERE, NEURO_LINEAR,
                      REPRO_CSO, REPRO_DE, REPRO_PSO, REPRO_RANDOM, REPRO_SBX_PM, Config,
                      NeuroDynamics, Plan, ServerStats, RveaError, check, lib)

__all__ = ["Run", "step_batch", "select", "gamma", "workspace_bytes", "RveaError",
           "DTLZ2_SPHERE", "DTLZ1_LINEAR", "DTLZ3_SPHERE", "DTLZ4_SPHERE", "NEURO_LINEAR",
           "REPRO_SBX_PM", "REPRO_DE", "REPRO_RANDOM", "REPRO_CSO", "REPRO_PSO",
           "lattice_size", "lattice_for"]


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def lattice_size(m: int, H: int) -> int:
    from math import comb
    return comb(H + m - 1, m - 1)


def lattice_for(m: int, n: int) -> int:
    """H of the largest lattice with at most n points: the reference vectors
    (and population size) of a run asked for n solutions."""
    return int(lib().rvea_lattice_for(int(m), int(n)))


def workspace_bytes(m: int, d: int, N: int) -> int:
    return int(lib().rvea_workspace_bytes(m, d, N))


class Run:
    """One optimisation run whose state stays resident on the device."""

    def __init__(self, m: int, d: int, N: int, H: int, problem: int = DTLZ2_SPHERE,
                 t_max: int = 100, alpha: float = 2.0, f_r: float = 0.1,
                 eta_c: float = 20.0, eta_m: float = 20.0, p_c: float = 1.0,
                 p_m: float = 1.0, lower: Optional[float] = None,
                 upper: Optional[float] = None, seed: int = 0, neuro=None,
                 reproduction: int = 0, de_F: float = 0.5, de_CR: float = 0.9,
                 cso_phi: float = 0.0, pso_w: float = 0.7298, pso_c1: float = 1.49618,
                 pso_c2: float = 1.49618, device=None, stream=None):
        self.device = torch.device("cuda" if device is None else device)
        if lower is None:
            lower = -1.0 if problem == NEURO_LINEAR else 0.0
        if upper is None:
            upper = 1.0
        self.m, self.d, self.N, self.H = m, d, N, H
        self.reproduction = reproduction
        self.problem, self.t_max = problem, t_max
        L = lib()
        cfg = Config(m, d, N, H, problem, t_max, alpha, f_r, eta_c, eta_m, p_c, p_m,
                     lower, upper, seed & 0xFFFFFFFFFFFFFFFF, None, reproduction, de_F, de_CR,
                     cso_phi, pso_w, pso_c1, pso_c2)
        self._neuro_keep = None
        if neuro is not None:
            A = np.ascontiguousarray(neuro["A"], dtype=np.float64)
            B = np.ascontiguousarray(neuro["B"], dtype=np.float64)
            nd = NeuroDynamics(A.shape[0], B.shape[1], neuro.get("h1", 64), neuro.get("h2", 64),
                               neuro.get("steps", 1000), neuro.get("sigma", 0.01),
                               A.ctypes.data_as(C.POINTER(C.c_double)),
                               B.ctypes.data_as(C.POINTER(C.c_double)), int(neuro.get("gemv", 0)))
            self._neuro_keep = (A, B, nd)
            cfg.neuro = C.pointer(nd)
        nbytes = int(L.rvea_workspace_bytes_ex(C.byref(cfg)))
        if nbytes == 0:
            raise RveaError(-1, "rvea_workspace_bytes_ex: invalid configuration")
        with torch.cuda.device(self.device):
            self._ws_raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws_raw.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        self.workspace_nbytes = nbytes
        self._h = C.c_void_p()
        with torch.cuda.device(self.device):
            check(L.rvea_init_ex(C.byref(cfg), C.c_void_p(self._ws_ptr), nbytes,
                                 C.c_void_p(_stream(stream)), C.byref(self._h)), "rvea_init_ex")

    # -- lifetime ------------------------------------------------------------
    def free(self) -> None:
        if self._h:
            lib().rvea_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def t(self) -> int:
        """Index of the next generation (1 after initialisation)."""
        return int(lib().rvea_generation(self._h))

    # -- generations ---------------------------------------------------------
    def step(self, generations: int = 1, stream=None) -> None:
        check(lib().rvea_step(self._h, int(generations), C.c_void_p(_stream(stream))), "rvea_step")

    def step_profiled(self, generations: int, stream=None):
        """Run generations with per-kernel CUDA events; returns the summed
        device milliseconds of (reproduction kernel, selection, finalize,
        gamma, the kernels finishing the children after reproduction)."""
        ms = (C.c_double * 5)()
        check(lib().rvea_step_profiled(self._h, int(generations), C.c_void_p(_stream(stream)),
                                       ms, 5), "rvea_step_profiled")
        return [float(x) for x in ms]

    def launches_per_generation(self, adapting: bool) -> int:
        """Kernel launches one generation enqueues (adapting: it rescales V)."""
        return int(lib().rvea_launches_per_generation(self._h, 1 if adapting else 0))

    def sync_status(self) -> None:
        check(lib().rvea_sync_status(self._h), "device status")

    # -- results -------------------------------------------------------------
    def population(self, out: Optional[torch.Tensor] = None, valid: Optional[torch.Tensor] = None,
                   stream=None):
        if out is None:
            out = torch.empty((self.N, self.d), dtype=torch.float32, device=self.device)
        if valid is None:
            valid = torch.empty(self.N, dtype=torch.uint8, device=self.device)
        check(lib().rvea_population(self._h, _ptr(out), _ptr(valid), C.c_void_p(_stream(stream))),
              "rvea_population")
        return out, valid

    def objectives(self, out: Optional[torch.Tensor] = None, valid: Optional[torch.Tensor] = None,
                   stream=None):
        if out is None:
            out = torch.empty((self.N, self.m), dtype=torch.float32, device=self.device)
        if valid is None:
            valid = torch.empty(self.N, dtype=torch.uint8, device=self.device)
        check(lib().rvea_objectives(self._h, _ptr(out), _ptr(valid), C.c_void_p(_stream(stream))),
              "rvea_objectives")
        return out, valid

    def igd(self, ref: torch.Tensor, stream=None) -> float:
        """Inverted generational distance of the current population against
        the reference points `ref` (n_ref x m float32 on the run's device)."""
        ref = ref.to(device=self.device, dtype=torch.float32).contiguous()
        if ref.dim() != 2 or ref.shape[1] != self.m:
            raise ValueError("ref must be n_ref x m")
        out = C.c_double()
        check(lib().rvea_igd(self._h, _ptr(ref), int(ref.shape[0]), C.byref(out),
                             C.c_void_p(_stream(stream))), "rvea_igd")
        return float(out.value)

    def hypervolume(self, ref, stream=None) -> float:
        """Hypervolume of the current population (m = 2 or 3) against the
        reference point `ref` (m values)."""
        if len(ref) != self.m:
            raise ValueError("ref must have m values")
        r = (C.c_double * self.m)(*[float(v) for v in ref])
        out = C.c_double()
        check(lib().rvea_hypervolume(self._h, r, C.byref(out), C.c_void_p(_stream(stream))),
              "rvea_hypervolume")
        return float(out.value)

    def export_state(self, stream=None) -> dict:
        dev = self.device
        X = torch.empty((self.N, self.d), dtype=torch.float32, device=dev)
        F = torch.empty((self.N, self.m), dtype=torch.float32, device=dev)
        valid = torch.empty(self.N, dtype=torch.uint8, device=dev)
        V = torch.empty((self.N, self.m), dtype=torch.float64, device=dev)
        g = torch.empty(self.N, dtype=torch.float64, device=dev)
        check(lib().rvea_export_state(self._h, _ptr(X), _ptr(F), _ptr(valid), _ptr(V), _ptr(g),
                                      C.c_void_p(_stream(stream))), "rvea_export_state")
        return dict(X=X, F=F, valid=valid, V=V, gamma=g, t=self.t)

    def import_state(self, X, F, valid, V, gamma, t: int, stream=None) -> None:
        dev = self.device
        X = torch.as_tensor(X, dtype=torch.float32, device=dev).contiguous()
        F = torch.as_tensor(F, dtype=torch.float32, device=dev).contiguous()
        valid = torch.as_tensor(valid, dtype=torch.uint8, device=dev).contiguous()
        V = torch.as_tensor(V, dtype=torch.float64, device=dev).contiguous()
        gamma = torch.as_tensor(gamma, dtype=torch.float64, device=dev).contiguous()
        check(lib().rvea_import_state(self._h, _ptr(X), _ptr(F), _ptr(valid), _ptr(V),
                                      _ptr(gamma), int(t), C.c_void_p(_stream(stream))),
              "rvea_import_state")

    def export_swarm(self, stream=None):
        """Velocities (N x d) and kept APDs (N) of a CSO or PSO run, by vector
        slot; for PSO also the personal bests (N x d) and their objectives
        (N x m), else None."""
        dev = self.device
        vel = torch.empty((self.N, self.d), dtype=torch.float32, device=dev)
        apd = torch.empty(self.N, dtype=torch.float32, device=dev)
        pso = self.reproduction == REPRO_PSO
        pb = torch.empty((self.N, self.d), dtype=torch.float32, device=dev) if pso else None
        fpb = torch.empty((self.N, self.m), dtype=torch.float32, device=dev) if pso else None
        check(lib().rvea_export_swarm(self._h, _ptr(vel), _ptr(apd), _ptr(pb), _ptr(fpb),
                                      C.c_void_p(_stream(stream))), "rvea_export_swarm")
        return vel, apd, pb, fpb

    def import_swarm(self, vel, apd, pbest=None, fpbest=None, stream=None) -> None:
        """Replace a CSO or PSO run's swarm state (after import_state)."""
        dev = self.device
        f32 = lambda a: None if a is None else torch.as_tensor(
            a, dtype=torch.float32, device=dev).contiguous()
        vel, apd, pbest, fpbest = f32(vel), f32(apd), f32(pbest), f32(fpbest)
        check(lib().rvea_import_swarm(self._h, _ptr(vel), _ptr(apd), _ptr(pbest), _ptr(fpbest),
                                      C.c_void_p(_stream(stream))), "rvea_import_swarm")

    def offspring(self, stream=None):
        X = torch.empty((self.N, self.d), dtype=torch.float32, device=self.device)
        F = torch.empty((self.N, self.m), dtype=torch.float32, device=self.device)
        check(lib().rvea_offspring(self._h, _ptr(X), _ptr(F), C.c_void_p(_stream(stream))),
              "rvea_offspring")
        return X, F

    def record_draws(self, enable: bool = True, stream=None) -> None:
        """Make later generations record their mating draws and mutation
        sites (rvea_record_draws)."""
        check(lib().rvea_record_draws(self._h, 1 if enable else 0, C.c_void_p(_stream(stream))),
              "rvea_record_draws")

    def last_draws(self, stream=None):
        """(parents (2 ceil(N/2),) int32 vector slots, counts (N,) int32 with -1
        for every site, sites (N, 32) int32) of the last generation."""
        P = (self.N + 1) // 2
        par = torch.empty(2 * P, dtype=torch.int32, device=self.device)
        sites = torch.empty((self.N, 33), dtype=torch.int32, device=self.device)
        check(lib().rvea_last_draws(self._h, _ptr(par), _ptr(sites), C.c_void_p(_stream(stream))),
              "rvea_last_draws")
        return par, sites[:, 0].contiguous(), sites[:, 1:].contiguous()

    def last_selection(self, stream=None):
        assoc = torch.empty(2 * self.N, dtype=torch.int32, device=self.device)
        surv = torch.empty(self.N, dtype=torch.int32, device=self.device)
        check(lib().rvea_last_selection(self._h, _ptr(assoc), _ptr(surv),
                                        C.c_void_p(_stream(stream))), "rvea_last_selection")
        return assoc, surv


def _plan_dict(pl) -> dict:
    return {"sel_mode": pl.sel_mode, "sel_per_sm": pl.sel_per_sm,
            "repro_staged": pl.repro_staged, "repro_us": pl.repro_us, "sel_us": pl.sel_us}


def get_plan(run: "Run") -> dict:
    """The run's kernel variants (see rvea_plan in include/rvea.h)."""
    pl = Plan()
    check(lib().rvea_get_plan(run.handle, C.byref(pl)), "rvea_get_plan")
    return _plan_dict(pl)


def set_plan(run: "Run", sel_mode: int, sel_per_sm: int = 8, repro_staged: int = 0,
             stream=None) -> None:
    """Choose the run's kernel variants; none changes its results."""
    pl = Plan(sel_mode, sel_per_sm, repro_staged, 0.0, 0.0)
    check(lib().rvea_set_plan(run.handle, C.byref(pl), C.c_void_p(_stream(stream))),
          "rvea_set_plan")


def autotune(run: "Run", use_cache: bool = True, stream=None) -> dict:
    """Time every kernel variant on the run's current generation (which is
    left unchanged) and keep the fastest; returns the plan and its times."""
    pl = Plan()
    check(lib().rvea_autotune(run.handle, C.c_void_p(_stream(stream)), int(use_cache),
                              C.byref(pl)), "rvea_autotune")
    return _plan_dict(pl)


class Batch:
    """A fixed set of runs stepped together: one batched generation captured
    as a CUDA graph, replayed per generation (rvea_batch_*)."""

    def __init__(self, runs: Sequence["Run"]):
        self.runs = list(runs)
        arr = (C.c_void_p * len(self.runs))(*[r.handle.value for r in self.runs])
        h = C.c_void_p()
        check(lib().rvea_batch_create(arr, len(self.runs), C.byref(h)), "rvea_batch_create")
        self._h = h

    def step(self, generations: int = 1, stream=None) -> None:
        check(lib().rvea_batch_step(self._h, int(generations), C.c_void_p(_stream(stream))),
              "rvea_batch_step")

    def launches_per_step(self) -> int:
        """Kernel launches of one batched generation (nodes of its graph)."""
        return int(lib().rvea_batch_launches_per_step(self._h))

    def step_profiled(self, generations: int, stream=None) -> list:
        """Device ms summed over `generations` per phase: reproduction, pruned
        association, full-scan association, finalize, gamma + tile tables."""
        ph = (C.c_double * 5)()
        check(lib().rvea_batch_step_profiled(self._h, int(generations),
                                             C.c_void_p(_stream(stream)), ph, 5),
              "rvea_batch_step_profiled")
        return list(ph)

    def free(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rvea_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """Serving loop with continuous batching (rvea_server_*): requests queue,
    are admitted between steps while their workspaces fit the arena (the HBM
    budget), and every step runs one generation of every live run."""

    def __init__(self, arena_bytes: int, max_live: int = 1 << 30, autotune: bool = True,
                 device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self._arena = torch.empty(int(arena_bytes) + 256, dtype=torch.uint8, device=self.device)
        base = (self._arena.data_ptr() + 255) & ~255
        h = C.c_void_p()
        check(lib().rvea_server_create(C.c_void_p(base), int(arena_bytes), int(max_live),
                                       int(autotune), C.byref(h)), "rvea_server_create")
        self._h = h
        self.meta = {}

    def submit(self, m: int, d: int, N: int, H: int, problem: int, generations: int,
               t_max: Optional[int] = None, alpha: float = 2.0, f_r: float = 0.1,
               eta_c: float = 20.0, eta_m: float = 20.0, p_c: float = 1.0, p_m: float = 1.0,
               seed: int = 0) -> int:
        cfg = Config(m, d, N, H, problem, generations if t_max is None else t_max, alpha, f_r,
                     eta_c, eta_m, p_c, p_m, 0.0, 1.0, seed & 0xFFFFFFFFFFFFFFFF, None)
        rid = C.c_int64()
        check(lib().rvea_server_submit(self._h, C.byref(cfg), int(generations), C.byref(rid)),
              "rvea_server_submit")
        self.meta[rid.value] = (m, d, N)
        return rid.value

    def step(self, stream=None) -> dict:
        st = ServerStats()
        check(lib().rvea_server_step(self._h, C.c_void_p(_stream(stream)), C.byref(st)),
              "rvea_server_step")
        return {"live": st.live, "queued": st.queued, "finished": st.finished,
                "admitted": st.admitted, "arena_used": st.arena_used,
                "generations": st.generations}

    def poll(self, cap: int = 4096) -> list:
        ids = (C.c_int64 * cap)()
        n = C.c_int()
        check(lib().rvea_server_poll(self._h, ids, cap, C.byref(n)), "rvea_server_poll")
        return [ids[q] for q in range(n.value)]

    def fetch(self, rid: int, stream=None):
        """(X (N, d), F (N, m), valid (N,)) on the device; releases the run."""
        m, d, N = self.meta.pop(rid)
        X = torch.empty((N, d), dtype=torch.float32, device=self.device)
        F = torch.empty((N, m), dtype=torch.float32, device=self.device)
        v = torch.empty(N, dtype=torch.uint8, device=self.device)
        check(lib().rvea_server_fetch(self._h, C.c_int64(rid), _ptr(X), _ptr(F), _ptr(v),
                                      C.c_void_p(_stream(stream))), "rvea_server_fetch")
        return X, F, v

    def free(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().rvea_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def step_batch(runs: Sequence[Run], stream=None) -> None:
    """One generation of every run in `runs`, one launch per phase."""
    arr = (C.c_void_p * len(runs))(*[r.handle.value for r in runs])
    check(lib().rvea_step_batch(arr, len(runs), C.c_void_p(_stream(stream))), "rvea_step_batch")


def select(F: torch.Tensor, valid: Optional[torch.Tensor], V: torch.Tensor, gam: torch.Tensor,
           t: int, t_max: int, alpha: float, scratch: Optional[torch.Tensor] = None, stream=None):
    """Environmental selection (Algorithm 1) of n solutions against r vectors.

    F (n, m) float32, valid (n,) uint8 or None, V (r, m) float32 unit rows,
    gam (r,) float32 -> (assoc (n,) int32, survivor (r,) int32)."""
    n, m = F.shape
    r = V.shape[0]
    dev = F.device
    F = F.contiguous().float()
    V = V.contiguous().float()
    gam = gam.contiguous().float()
    if valid is not None:
        valid = valid.contiguous().to(torch.uint8)
    need = int(lib().rvea_select_scratch_bytes(n, r, m))
    if scratch is None:
        raw = torch.empty(need + 256, dtype=torch.uint8, device=dev)
        sp = (raw.data_ptr() + 255) & ~255
    else:
        raw = scratch
        sp = scratch.data_ptr()
    assoc = torch.empty(n, dtype=torch.int32, device=dev)
    surv = torch.empty(r, dtype=torch.int32, device=dev)
    check(lib().rvea_select(m, n, _ptr(F), _ptr(valid), r, _ptr(V), _ptr(gam), int(t),
                            int(t_max), float(alpha), _ptr(assoc), _ptr(surv), C.c_void_p(sp),
                            need, C.c_void_p(_stream(stream))), "rvea_select")
    torch.cuda.current_stream(dev).synchronize() if stream is None else None
    del raw
    return assoc, surv


def gamma(V: torch.Tensor, stream=None) -> torch.Tensor:
    """Minimum angle from each unit row of V (r, m) float64 to the others."""
    V = V.contiguous().double()
    r, m = V.shape
    g = torch.empty(r, dtype=torch.float64, device=V.device)
    check(lib().rvea_gamma(m, r, _ptr(V), _ptr(g), C.c_void_p(_stream(stream))), "rvea_gamma")
    return g
