"""Thin PyTorch binding of libdg (argument marshalling only).

PyTorch provides device memory and streams; every step of the solver runs in
libdg's sm_103a kernels behind the C ABI of ``include/dg.h``.  The names follow
the C ABI: :func:`plan` (host build of the BDD arena), :meth:`Plan.bind`
(device upload), :meth:`Arena.init_lambda`, :meth:`Arena.iterate`,
:meth:`Arena.min_marginals`, :meth:`Arena.lower_bound`,
:meth:`Arena.lb_seed`, :meth:`Arena.backward` and the graph calls.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check, dg_options, dg_rows, dg_sizes, dg_stats


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


def make_options(tile_nodes=0, tile_slots=0, block_threads=0, renorm_every=0, omega=0.0, num_threads=0,
                 host_mb_limit=0, chunk_rows=0, group_ratio_pct=0, long_lanes=0):
    o = dg_options()
    o.long_lanes = int(long_lanes)
    o.host_mb_limit = int(host_mb_limit)
    o.chunk_rows = int(chunk_rows)
    o.group_ratio_pct = int(group_ratio_pct)
    o.tile_nodes = int(tile_nodes)
    o.tile_slots = int(tile_slots)
    o.block_threads = int(block_threads)
    o.renorm_every = int(renorm_every)
    o.omega = float(omega)
    o.num_threads = int(num_threads)
    return o


class Plan:
    """Host layout of a batch of binary programs (``dg_plan``)."""

    def __init__(self, rows: dict, options: dg_options | None = None):
        lib = _lib.load()
        self._keep = dict(
            row_ptr=np.ascontiguousarray(rows["row_ptr"], dtype=np.int64),
            col=np.ascontiguousarray(rows["col"], dtype=np.int32),
            coef=np.ascontiguousarray(rows["coef"], dtype=np.int32),
            sense=np.ascontiguousarray(rows["sense"], dtype=np.int8),
            rhs=np.ascontiguousarray(rows["rhs"], dtype=np.int32),
            c=np.ascontiguousarray(rows["c"], dtype=np.float64),
        )
        r = dg_rows()
        if rows.get("inst_row_ptr") is not None:
            self._keep["irp"] = np.ascontiguousarray(rows["inst_row_ptr"], dtype=np.int64)
            self._keep["ivp"] = np.ascontiguousarray(rows["inst_var_ptr"], dtype=np.int32)
            r.num_inst = len(self._keep["irp"]) - 1
            r.inst_row_ptr = _ptr(self._keep["irp"])
            r.inst_var_ptr = _ptr(self._keep["ivp"])
        else:
            r.num_inst = 1
        k = self._keep
        r.n = int(rows["n"])
        r.m = len(k["row_ptr"]) - 1
        r.row_ptr, r.col, r.coef = _ptr(k["row_ptr"]), _ptr(k["col"]), _ptr(k["coef"])
        r.sense, r.rhs, r.c = _ptr(k["sense"]), _ptr(k["rhs"]), _ptr(k["c"])
        self.options = options if options is not None else make_options()
        h = ctypes.c_void_p()
        sz = dg_sizes()
        check(lib.dg_plan(ctypes.byref(r), ctypes.byref(self.options), ctypes.byref(h), ctypes.byref(sz)), "dg_plan")
        self._h = h
        self.sizes = sz
        self.n = sz.n
        self.m = sz.m
        self.num_slots = sz.num_slots
        self.num_inst = sz.num_inst
        sm = np.zeros(sz.num_slots, np.int64)
        check(lib.dg_slot_map(h, _ptr(sm)), "dg_slot_map")
        self.slot_to_csr = sm

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib._lib is not None:
            _lib._lib.dg_plan_free(self._h)
            self._h = None

    def bdd(self, j: int):
        """(level_start, lo, hi) of row j as built (children as ranks, -2 bottom, -1 top)."""
        lib = _lib.load()
        nn = ctypes.c_int32()
        check(lib.dg_bdd_export(self._h, int(j), None, None, None, ctypes.byref(nn)), "dg_bdd_export")
        k = int(self._keep["row_ptr"][j + 1] - self._keep["row_ptr"][j])
        ls = np.zeros(k + 1, np.int32)
        lo = np.zeros(nn.value, np.int32)
        hi = np.zeros(nn.value, np.int32)
        check(lib.dg_bdd_export(self._h, int(j), _ptr(ls), _ptr(lo), _ptr(hi), ctypes.byref(nn)), "dg_bdd_export")
        return ls, lo, hi

    def validate(self):
        """dg_plan_validate: structural invariants of the arena image (raises on a violation)."""
        check(_lib.load().dg_plan_validate(self._h), "dg_plan_validate")

    def launch_groups(self):
        """[(tile0, tile1, per-warp shared bytes, stream)] of the sweep launches."""
        out = []
        for g in range(int(self.sizes.num_launch_groups)):
            v = [ctypes.c_int32() for _ in range(4)]
            check(_lib.load().dg_launch_group(self._h, g, *[ctypes.byref(x) for x in v]), "dg_launch_group")
            out.append(tuple(x.value for x in v))
        return out

    def bind(self, device=None, stream=None) -> "Arena":
        return Arena(self, device, stream)


def plan(rows: dict, **opts) -> Plan:
    return Plan(rows, make_options(**opts))


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Arena:
    """A bound arena: device layout plus the state-vector helpers."""

    def __init__(self, plan: Plan, device=None, stream=None):
        lib = _lib.load()
        self.plan = plan
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = int(plan.sizes.arena_bytes)
        self.buffer = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.buffer.data_ptr()
        self._off = (-base) % 256
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(lib.dg_bind(plan._h, ctypes.c_void_p(base + self._off), nbytes, _stream_handle(stream),
                              ctypes.byref(h)), "dg_bind")
        self._h = h
        st = dg_stats()
        check(lib.dg_get_stats(h, ctypes.byref(st)), "dg_get_stats")
        self.stats = st
        self.num_slots = plan.num_slots
        self.n, self.m, self.num_inst = plan.n, plan.m, plan.num_inst
        sm = plan.slot_to_csr
        self.slot_to_csr = torch.from_numpy(sm).to(self.device)
        self.real = self.slot_to_csr >= 0
        self.csr_to_slot = torch.empty(int(plan.sizes.num_lambda), dtype=torch.int64, device=self.device)
        self.csr_to_slot[self.slot_to_csr[self.real]] = torch.nonzero(self.real).flatten()
        self.options = plan.options

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib._lib is not None:
            _lib._lib.dg_destroy(self._h)
            self._h = None

    def slot_instance(self):
        """Instance of every arena slot (padding: 0), for per-instance scaling."""
        if getattr(self, "_slot_inst", None) is None:
            rp = self.plan._keep["row_ptr"]
            irp = self.plan._keep.get("irp")
            sm = self.plan.slot_to_csr
            rows = np.searchsorted(rp, np.maximum(sm, 0), side="right") - 1
            inst = np.zeros_like(rows) if irp is None else np.searchsorted(irp, rows, side="right") - 1
            inst[sm < 0] = 0
            self._slot_inst = torch.from_numpy(inst.astype(np.int64)).to(self.device)
        return self._slot_inst

    # -- marshalling helpers (index permutations only) ---------------------
    def zeros(self, dtype=torch.float32):
        return torch.zeros(self.num_slots, dtype=dtype, device=self.device)

    def to_csr(self, x: torch.Tensor) -> torch.Tensor:
        """Arena-order vector -> CSR-order vector (drops padding)."""
        return x[self.csr_to_slot]

    def from_csr(self, x, dtype=torch.float32) -> torch.Tensor:
        """CSR-order vector -> arena order (padding 0)."""
        x = torch.as_tensor(x, device=self.device).to(dtype)
        out = torch.zeros(self.num_slots, dtype=dtype, device=self.device)
        out[self.csr_to_slot] = x
        return out

    # -- solver --------------------------------------------------------------
    def init_lambda(self, stream=None):
        lam, M = self.zeros(), self.zeros()
        check(_lib.load().dg_init_lambda(self._h, _stream_handle(stream), _ptr(lam), _ptr(M)), "dg_init_lambda")
        return lam, M

    def _opts(self, **kw):
        if not kw:
            return self.options
        o = dg_options()
        ctypes.pointer(o)[0] = self.options
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    def iterate(self, lam, M, omega=None, alpha=None, iters=1, lb=False, stream=None, **opt):
        """Runs ``iters`` iterations of Alg. 1 in place; returns the per-instance
        bound (float64 tensor) if ``lb``."""
        mode = 0 if omega is None else 1
        if mode == 1 and alpha is None:
            raise ValueError("per-slot omega needs per-slot alpha")
        lb_out = torch.zeros(self.num_inst, dtype=torch.float64, device=self.device) if lb else None
        o = self._opts(**opt)
        check(_lib.load().dg_iterate(self._h, _stream_handle(stream), _ptr(lam), _ptr(M), _ptr(omega), _ptr(alpha),
                                     mode, int(iters), _ptr(lb_out), ctypes.byref(o)), "dg_iterate")
        return lb_out

    # building blocks of iterate (one kernel each), for per-kernel timing
    def sum_M(self, M, lam=None, alpha=None, renorm=False, stream=None):
        mode = 0 if alpha is None else 1
        check(_lib.load().dg_sum_M(self._h, _stream_handle(stream), _ptr(M), _ptr(lam), _ptr(alpha), mode,
                                   int(bool(renorm))), "dg_sum_M")

    def sweep(self, lam, M, forward, omega=None, alpha=None, energy=False, stream=None, costs_out=False,
              costs_in=False):
        """dg_sweep; costs_out / costs_in are DG_SWEEP_COSTS_OUT / DG_SWEEP_COSTS_IN."""
        mode = 0 if omega is None else 1
        flags = (_lib.DG_SWEEP_ENERGY if energy else 0) | (_lib.DG_SWEEP_COSTS_OUT if costs_out else 0) | \
            (_lib.DG_SWEEP_COSTS_IN if costs_in else 0)
        check(_lib.load().dg_sweep(self._h, _stream_handle(stream), _ptr(lam), _ptr(M), _ptr(omega), _ptr(alpha),
                                   mode, int(bool(forward)), flags, ctypes.byref(self.options)),
              "dg_sweep")

    def bound_from_energies(self, lb_out, stream=None):
        check(_lib.load().dg_bound_from_energies(self._h, _stream_handle(stream), _ptr(lb_out)),
              "dg_bound_from_energies")

    def iterate_launches(self, iters, lb=False):
        return int(_lib.load().dg_iterate_launches(self._h, int(iters), int(bool(lb)), ctypes.byref(self.options)))

    def min_marginals(self, lam, stream=None):
        m0, m1 = self.zeros(), self.zeros()
        check(_lib.load().dg_min_marginals(self._h, _stream_handle(stream), _ptr(lam), _ptr(m0), _ptr(m1)),
              "dg_min_marginals")
        return m0, m1

    def lower_bound(self, lam, M, energies=False, stream=None):
        lb = torch.zeros(self.num_inst, dtype=torch.float64, device=self.device)
        E = torch.zeros(self.m, dtype=torch.float32, device=self.device) if energies else None
        check(_lib.load().dg_lower_bound(self._h, _stream_handle(stream), _ptr(lam), _ptr(M), _ptr(lb), _ptr(E)),
              "dg_lower_bound")
        return (lb, E) if energies else lb

    def lower_bound_noalloc(self, lam, M, out=None, stream=None):
        """dg_lower_bound_noalloc: the bound with libdg's static scratch; ``out``
        (float64[num_inst] on the device) may be passed in by callers that
        manage their own memory."""
        lb = out if out is not None else torch.zeros(self.num_inst, dtype=torch.float64, device=self.device)
        check(_lib.load().dg_lower_bound_noalloc(self._h, _stream_handle(stream), _ptr(lam), _ptr(M), _ptr(lb)),
              "dg_lower_bound_noalloc")
        return lb

    def lb_seed(self, lam, M, stream=None):
        gl, gM = self.zeros(), self.zeros()
        self.lb_seed_into(lam, M, gl, gM, stream)
        return gl, gM

    def lb_seed_into(self, lam, M, g_lam, g_M, stream=None):
        check(_lib.load().dg_lb_seed(self._h, _stream_handle(stream), _ptr(lam), _ptr(M), _ptr(g_lam), _ptr(g_M)),
              "dg_lb_seed")

    def smoothed_dual(self, lam, a, stream=None):
        """(E_a per row, marginals per slot) of the smoothed subproblems."""
        E = torch.zeros(self.m, dtype=torch.float32, device=self.device)
        mg = self.zeros()
        check(_lib.load().dg_smoothed_dual(self._h, _stream_handle(stream), _ptr(lam), float(a), _ptr(E), _ptr(mg)),
              "dg_smoothed_dual")
        return E, mg

    # -- DOGE-Train's updates around the solver (eq. 2, Alg. 3) ------------
    def nonparam_update(self, lam, theta, stream=None):
        check(_lib.load().dg_nonparam_update(self._h, _stream_handle(stream), _ptr(lam), _ptr(theta)),
              "dg_nonparam_update")

    def nonparam_backward(self, g_lam, stream=None):
        g = self.zeros()
        check(_lib.load().dg_nonparam_backward(self._h, _stream_handle(stream), _ptr(g_lam), _ptr(g)),
              "dg_nonparam_backward")
        return g

    def param_transform(self, alpha_hat, omega_hat, theta_hat, stream=None):
        outs = [self.zeros() if x is not None else None for x in (alpha_hat, omega_hat, theta_hat)]
        check(_lib.load().dg_param_transform(self._h, _stream_handle(stream), _ptr(alpha_hat), _ptr(omega_hat),
                                             _ptr(theta_hat), *[_ptr(o) for o in outs]), "dg_param_transform")
        return tuple(outs)

    def param_transform_backward(self, alpha, omega, g_alpha, g_omega, g_theta, stream=None):
        outs = [self.zeros() if g is not None else None for g in (g_alpha, g_omega, g_theta)]
        check(_lib.load().dg_param_transform_backward(self._h, _stream_handle(stream), _ptr(alpha), _ptr(omega),
                                                      _ptr(g_alpha), _ptr(g_omega), _ptr(g_theta),
                                                      *[_ptr(o) for o in outs]), "dg_param_transform_backward")
        return tuple(outs)

    def graph(self, lam, M, omega=None, alpha=None, iters=1, lb_out=None, stream=None, **opt):
        return Graph(self, lam, M, omega, alpha, iters, lb_out, stream, self._opts(**opt))

    def backward_workspace_bytes(self, iters, ckpt_every):
        return int(_lib.load().dg_backward_workspace_bytes(self._h, int(iters), int(ckpt_every)))

    def backward(self, lam0, M0, omega, alpha, iters, ckpt_every, g_lamT, g_MT, stream=None, workspace=None):
        """Alg. 2 through ``iters`` iterations; returns (g_lam0, g_M0, g_omega, g_alpha)."""
        outs = [self.zeros() for _ in range(4)]
        self.backward_into(lam0, M0, omega, alpha, iters, ckpt_every, g_lamT, g_MT, outs, workspace, stream)
        return tuple(outs)

    def backward_into(self, lam0, M0, omega, alpha, iters, ckpt_every, g_lamT, g_MT, outs, workspace=None,
                      stream=None):
        mode = 0 if omega is None else 1
        ws_bytes = self.backward_workspace_bytes(iters, ckpt_every)
        if workspace is None:
            workspace = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=self.device)
        check(_lib.load().dg_backward(self._h, _stream_handle(stream), _ptr(lam0), _ptr(M0), _ptr(omega),
                                      _ptr(alpha), mode, int(iters), int(ckpt_every), _ptr(g_lamT), _ptr(g_MT),
                                      *[_ptr(o) for o in outs], _ptr(workspace), int(workspace.numel()),
                                      ctypes.byref(self.options)), "dg_backward")


    def iterate_checkpointed(self, lam, M, omega=None, alpha=None, iters=1, ckpt_every=10, workspace=None, lb=False,
                             stream=None, **opt):
        """``iterate`` in place that also keeps the checkpoints ``backward_checkpointed``
        needs; returns (workspace, bound or None)."""
        mode = 0 if omega is None else 1
        if mode == 1 and alpha is None:
            raise ValueError("per-slot omega needs per-slot alpha")
        ws_bytes = self.backward_workspace_bytes(iters, ckpt_every)
        if workspace is None:
            workspace = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=self.device)
        lb_out = torch.zeros(self.num_inst, dtype=torch.float64, device=self.device) if lb else None
        o = self._opts(**opt)
        check(_lib.load().dg_iterate_checkpointed(self._h, _stream_handle(stream), _ptr(lam), _ptr(M), _ptr(omega),
                                                  _ptr(alpha), mode, int(iters), int(ckpt_every), _ptr(workspace),
                                                  int(workspace.numel()), _ptr(lb_out), ctypes.byref(o)),
              "dg_iterate_checkpointed")
        return workspace, lb_out

    def backward_checkpointed(self, omega, alpha, iters, ckpt_every, g_lamT, g_MT, workspace, outs=None,
                              stream=None):
        """Alg. 2 from the checkpoints of ``iterate_checkpointed``; returns
        (g_lam0, g_M0, g_omega, g_alpha)."""
        mode = 0 if omega is None else 1
        outs = outs if outs is not None else [self.zeros() for _ in range(4)]
        check(_lib.load().dg_backward_checkpointed(self._h, _stream_handle(stream), _ptr(omega), _ptr(alpha), mode,
                                                   int(iters), int(ckpt_every), _ptr(g_lamT), _ptr(g_MT),
                                                   *[_ptr(o) for o in outs], _ptr(workspace), int(workspace.numel()),
                                                   ctypes.byref(self.options)), "dg_backward_checkpointed")
        return tuple(outs)


def wait(stream=None, timeout_ms=1000):
    """dg_wait: bounded host wait for the stream's work; returns the status."""
    return int(_lib.load().dg_wait(_stream_handle(stream), int(timeout_ms)))


class DualIterate(torch.autograd.Function):
    """(lam0, M0, omega, alpha) -> (lam_T, M_T) through ``iters`` iterations of
    Alg. 1 (dg_iterate_checkpointed, which keeps (lam, M) every ``ckpt_every``
    iterations); backward is Alg. 2 from those checkpoints
    (dg_backward_checkpointed).  ``omega``/``alpha`` None selects
    the plain method (scalar omega of the arena's options, alpha = 1/|J_i|)."""

    @staticmethod
    def forward(ctx, lam0, M0, omega, alpha, arena, iters, ckpt_every):
        lam, M = lam0.detach().clone(), M0.detach().clone()
        om = omega.detach() if omega is not None else None
        al = alpha.detach() if alpha is not None else None
        # the checkpoints of the backward pass are taken here, on the way
        ctx.workspace, _ = arena.iterate_checkpointed(lam, M, om, al, iters=iters, ckpt_every=ckpt_every)
        ctx.arena, ctx.iters, ctx.ckpt = arena, int(iters), int(ckpt_every)
        ctx.has_params = omega is not None
        ctx.save_for_backward(om, al)
        return lam, M

    @staticmethod
    def backward(ctx, g_lam, g_M):
        om, al = ctx.saved_tensors
        A = ctx.arena
        g_lam = A.zeros() if g_lam is None else g_lam.contiguous().float()
        g_M = A.zeros() if g_M is None else g_M.contiguous().float()
        # the per-slot parameter gradients only when autograd wants them
        need_w = ctx.has_params and ctx.needs_input_grad[2]
        need_a = ctx.has_params and ctx.needs_input_grad[3]
        outs = [A.zeros(), A.zeros(), A.zeros() if need_w else None, A.zeros() if need_a else None]
        gl0, gM0, gw, ga = A.backward_checkpointed(om, al, ctx.iters, ctx.ckpt, g_lam, g_M, ctx.workspace, outs=outs)
        ctx.workspace = None
        return gl0, gM0, gw, ga, None, None, None


class LowerBound(torch.autograd.Function):
    """Per-instance lower bound (dg_lower_bound) with the loss gradient of
    eq. (3) plus the unary term (dg_lb_seed) as backward."""

    @staticmethod
    def forward(ctx, lam, M, arena):
        ctx.arena = arena
        ctx.save_for_backward(lam.detach(), M.detach())
        return arena.lower_bound(lam.detach(), M.detach())

    @staticmethod
    def backward(ctx, g):
        lam, M = ctx.saved_tensors
        A = ctx.arena
        gl, gM = A.lb_seed(lam, M)
        if A.num_inst == 1:
            w = g.float()[0]
            return gl * w, gM * w, None
        scale = g.float()[A.slot_instance()]
        return gl * scale, gM * scale, None


class NonParamUpdate(torch.autograd.Function):
    """lam + theta - mean_{J_i} theta (eq. 2), on the device."""

    @staticmethod
    def forward(ctx, lam, theta, arena):
        ctx.arena = arena
        out = lam.detach().clone()
        arena.nonparam_update(out, theta.detach().contiguous())
        return out

    @staticmethod
    def backward(ctx, g):
        g = g.contiguous().float()
        return g, ctx.arena.nonparam_backward(g), None


class ParamTransform(torch.autograd.Function):
    """(alpha_hat, omega_hat, theta_hat) -> (softmax over J_i, sigmoid, centred)
    as in Alg. 3, on the device."""

    @staticmethod
    def forward(ctx, alpha_hat, omega_hat, theta_hat, arena):
        ctx.arena = arena
        a, w, t = arena.param_transform(alpha_hat.detach().contiguous(), omega_hat.detach().contiguous(),
                                        theta_hat.detach().contiguous())
        ctx.save_for_backward(a, w)
        return a, w, t

    @staticmethod
    def backward(ctx, ga, gw, gt):
        a, w = ctx.saved_tensors
        A = ctx.arena
        ga = A.zeros() if ga is None else ga.contiguous().float()
        gw = A.zeros() if gw is None else gw.contiguous().float()
        gt = A.zeros() if gt is None else gt.contiguous().float()
        gah, gwh, gth = A.param_transform_backward(a, w, ga, gw, gt)
        return gah, gwh, gth, None


class Graph:
    """CUDA graph of ``iters`` iterations on fixed buffers (dg_graph_create)."""

    def __init__(self, arena, lam, M, omega, alpha, iters, lb_out, stream, opts):
        self.arena = arena
        self._keep = (lam, M, omega, alpha, lb_out)
        mode = 0 if omega is None else 1
        h = ctypes.c_void_p()
        self._stream = stream if stream is not None else torch.cuda.Stream(device=arena.device)
        check(_lib.load().dg_graph_create(arena._h, ctypes.c_void_p(self._stream.cuda_stream), _ptr(lam), _ptr(M),
                                          _ptr(omega), _ptr(alpha), mode, int(iters), _ptr(lb_out),
                                          ctypes.byref(opts), ctypes.byref(h)), "dg_graph_create")
        self._h = h

    def replay(self, stream=None):
        check(_lib.load().dg_graph_replay(self._h, _stream_handle(stream)), "dg_graph_replay")

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib._lib is not None:
            _lib._lib.dg_graph_destroy(self._h)
            self._h = None
