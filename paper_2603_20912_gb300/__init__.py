"""Python binding of libladder.so (the GB300 particle-particle ladder library).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI declared in ``include/ladder.h``.  PyTorch supplies
device memory and streams.  There is no CPU fallback -- if the library is not
built, importing the binding raises.

The function names mirror the C ABI::

    plan = ladder_plan(no, nv, nchol, precision=LADDER_FP64, nslices=0, ws_budget_bytes=0, device=0)
    ws = plan.workspace()                       # torch.uint8 device tensor
    ladder_apply(plan, L, t2, R, ws)            # R += sum_cd (ac|bd) t2[i,j,c,d]
    E = ladder_energy(plan, t2, R)              # E_L as a Python float
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build_mod

LADDER_OK = 0
LADDER_ERR_ARG = 1
LADDER_ERR_BUDGET = 2
LADDER_ERR_CUDA = 3
LADDER_ERR_UNSUPPORTED = 4
LADDER_ERR_TIMEOUT = 5
LADDER_ERR_NUMERIC = 6
LADDER_ERR_BOUNDS = 7

LADDER_FP64 = 0
LADDER_EMU_BF16 = 1
LADDER_EMU_INT8 = 2

LADDER_KERNEL_PREP = 0
LADDER_KERNEL_ERI = 1
LADDER_KERNEL_LADDER = 2
LADDER_KERNEL_FINISH = 3
LADDER_KERNEL_COMBINE = 4
LADDER_KERNEL_FACT_W = 5
LADDER_KERNEL_FACT_R = 6
LADDER_KERNEL_FUSED = 7

LADDER_PATH_ERI = 0
LADDER_PATH_FACTORISED = 1
LADDER_PATH_FUSED = 2

# LADDER_CHECKED_LIBRARY=1 loads the index-checked build (build.build(check=True)) instead.
LIB_PATH = _build_mod.LIB_CHECK if os.environ.get("LADDER_CHECKED_LIBRARY") == "1" else _build_mod.LIB

_lib = None


class LadderError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {ladder_strerror(status)} (status {status})")


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libladder.so is not built ({LIB_PATH}); run "
                          "`python -m paper_2603_20912_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, sz, ci = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
    pint = ctypes.POINTER(ci)
    lib.ladder_plan.argtypes = [ctypes.POINTER(vp), ci, ci, ci, ci, ci, sz, ci]
    lib.ladder_plan.restype = ci
    lib.ladder_plan_set_form.argtypes = [vp, ci]
    lib.ladder_plan_set_form.restype = ci
    lib.ladder_plan_get_form.argtypes = [vp]
    lib.ladder_plan_get_form.restype = ci
    lib.ladder_form_model.argtypes = [ci, ci, ci, ci]
    lib.ladder_form_model.restype = ci
    lib.ladder_plan_set_pbatch.argtypes = [vp, ci]
    lib.ladder_plan_set_pbatch.restype = ci
    lib.ladder_plan_get_pbatch.argtypes = [vp]
    lib.ladder_plan_get_pbatch.restype = ci
    lib.ladder_plan_set_eri_chunk.argtypes = [vp, ci]
    lib.ladder_plan_set_eri_chunk.restype = ci
    lib.ladder_plan_eri_chunk.argtypes = [vp, vp, vp]
    lib.ladder_plan_eri_chunk.restype = ci
    lib.ladder_plan_set_ladder_tile.argtypes = [vp, ci]
    lib.ladder_plan_set_ladder_tile.restype = ci
    lib.ladder_plan_get_ladder_tile.argtypes = [vp]
    lib.ladder_plan_get_ladder_tile.restype = ci
    lib.ladder_plan_set_path.argtypes = [vp, ci]
    lib.ladder_plan_set_path.restype = ci
    lib.ladder_plan_get_path.argtypes = [vp]
    lib.ladder_plan_get_path.restype = ci
    lib.ladder_path_model.argtypes = [ci, ci, ci, ci]
    lib.ladder_path_model.restype = ci
    lib.ladder_batched_schedule.argtypes = [vp, ci, pint]
    lib.ladder_batched_schedule.restype = ci
    lib.ladder_watchdog_selftest.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_double), vp]
    lib.ladder_watchdog_selftest.restype = ci
    lib.ladder_plan_shard.argtypes = [vp, ci, ci]
    lib.ladder_plan_shard.restype = ci
    lib.ladder_shard_blocks.argtypes = [ci, ctypes.POINTER(ctypes.c_longlong), ci, pint]
    lib.ladder_shard_blocks.restype = ci
    lib.ladder_plan_set_blocks.argtypes = [vp, ci, ci]
    lib.ladder_plan_set_blocks.restype = ci
    lib.ladder_workspace_bytes.argtypes = [vp]
    lib.ladder_workspace_bytes.restype = sz
    lib.ladder_plan_describe.argtypes = [vp, pint, pint, pint, pint, pint, pint]
    lib.ladder_plan_describe.restype = ci
    lib.ladder_apply.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.ladder_apply.restype = ci
    lib.ladder_apply_host.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.ladder_apply_host.restype = ci
    lib.ladder_host_staging_bytes.argtypes = [vp]
    lib.ladder_host_staging_bytes.restype = sz
    lib.ladder_energy.argtypes = [vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double), vp]
    lib.ladder_energy.restype = ci
    lib.ladder_plan_batched.argtypes = [ctypes.POINTER(vp), ci, pint, pint, pint, ci, ci, sz, ci]
    lib.ladder_plan_batched.restype = ci
    lib.ladder_apply_batched.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp]
    lib.ladder_apply_batched.restype = ci
    lib.ladder_tune_batched.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp, pint]
    lib.ladder_tune_batched.restype = ci
    lib.ladder_last_status.argtypes = [vp, vp]
    lib.ladder_last_status.restype = ci
    lib.ladder_plan_destroy.argtypes = [vp]
    lib.ladder_plan_destroy.restype = None
    lib.ladder_strerror.argtypes = [ci]
    lib.ladder_strerror.restype = ctypes.c_char_p
    lib.ladder_plan_dry.argtypes = [ci, ci, ci, ci, ci, sz, ci, ci, ci, pint, pint, ctypes.POINTER(sz), ci, pint,
                                    pint]
    lib.ladder_plan_dry.restype = ci
    lib.ladder_plan_shard_dry.argtypes = [ci, ci, ci, ci, ci, sz, ci, ci, ci, pint, pint, ctypes.POINTER(sz), ci,
                                          pint, pint]
    lib.ladder_plan_shard_dry.restype = ci
    lib.ladder_plan_set_wait_limit.argtypes = [vp, ctypes.c_double]
    lib.ladder_plan_set_wait_limit.restype = ci
    lib.ladder_plan_get_wait_limit.argtypes = [vp]
    lib.ladder_plan_get_wait_limit.restype = ctypes.c_double
    lib.ladder_plan_set_timing.argtypes = [vp, ci]
    lib.ladder_plan_set_timing.restype = ci
    lib.ladder_plan_timing.argtypes = [vp, ci, ctypes.POINTER(ctypes.c_float), pint, ci]
    lib.ladder_plan_timing.restype = ci
    lib.ladder_energy_noalloc.argtypes = [ci, ci, vp, vp, vp, vp]
    lib.ladder_energy_noalloc.restype = ci
    lib.ladder_flops.argtypes = [ci, ci, ci]
    lib.ladder_flops.restype = ctypes.c_double
    _lib = lib
    return lib


def lib():
    """The loaded ctypes library (raises if it is not built)."""
    return _load()


def ladder_strerror(status: int) -> str:
    return _load().ladder_strerror(int(status)).decode()


def ladder_flops(no: int, nv: int, nchol: int) -> float:
    return float(_load().ladder_flops(no, nv, nchol))


def _check(status: int, what: str):
    if status != LADDER_OK:
        raise LadderError(status, what)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """Owns a ladder_plan_t handle."""

    def __init__(self, handle, no=None, nv=None, nchol=None, device=0, batched_shapes=None):
        self._h = handle
        self.no, self.nv, self.nchol = no, nv, nchol
        self.device = device
        self.batched_shapes = batched_shapes

    @property
    def handle(self):
        return self._h

    def workspace_bytes(self) -> int:
        return int(_load().ladder_workspace_bytes(self._h))

    def workspace(self):
        import torch
        # Round up so the tensor start (torch: 512-byte aligned) stays usable.
        return torch.empty(max(self.workspace_bytes(), 256), dtype=torch.uint8, device=f"cuda:{self.device}")

    def host_staging_bytes(self) -> int:
        return int(_load().ladder_host_staging_bytes(self._h))

    def host_staging(self):
        """A device buffer of host_staging_bytes() bytes for ladder_apply_host."""
        import torch
        return torch.empty(max(self.host_staging_bytes(), 256), dtype=torch.uint8, device=f"cuda:{self.device}")

    def describe(self) -> dict:
        vals = [ctypes.c_int() for _ in range(6)]
        _check(_load().ladder_plan_describe(self._h, *[ctypes.byref(v) for v in vals]), "ladder_plan_describe")
        keys = ["n_a", "n_b", "n_block_pairs", "max_pairs_per_block", "nslices", "precision"]
        return {k: v.value for k, v in zip(keys, vals)}

    def set_blocks(self, n_a: int, n_b: int):
        _check(_load().ladder_plan_set_blocks(self._h, int(n_a), int(n_b)), "ladder_plan_set_blocks")

    def form(self) -> int:
        return int(_load().ladder_plan_get_form(self._h))

    def pbatch(self) -> int:
        return int(_load().ladder_plan_get_pbatch(self._h))

    def set_pbatch(self, pb: int):
        """Slice the Cholesky vectors pb at a time (0: all at once); see ladder_plan_set_pbatch."""
        _check(_load().ladder_plan_set_pbatch(self._h, int(pb)), "ladder_plan_set_pbatch")

    def set_eri_chunk(self, blocks: int):
        """Longest exact K chunk of the emulated ERI in blocks of 1024 (1..4); see ladder_plan_set_eri_chunk."""
        _check(_load().ladder_plan_set_eri_chunk(self._h, int(blocks)), "ladder_plan_set_eri_chunk")

    def eri_chunk(self, ws, stream=None) -> int:
        """Chunk length (Cholesky vectors) the last ladder_apply with this workspace chose."""
        return int(_load().ladder_plan_eri_chunk(self._h, ctypes.c_void_p(ws.data_ptr()), _stream_handle(stream)))

    def ladder_tile(self) -> int:
        return int(_load().ladder_plan_get_ladder_tile(self._h))

    def set_ladder_tile(self, bn: int):
        """Pairs per column tile of the one-SM emulated ladder (multiple of 16 in [16, 96])."""
        _check(_load().ladder_plan_set_ladder_tile(self._h, int(bn)), "ladder_plan_set_ladder_tile")

    def batched_choice(self) -> dict:
        """The tile width a batched plan holds (after ladder_tune_batched: the tuner's choice)."""
        return {"ladder_tile": self.ladder_tile()}

    def path(self) -> int:
        return int(_load().ladder_plan_get_path(self._h))

    def set_path(self, path: int):
        """0: rebuild (ac|bd) per block pair; 1: factorised sum_P L_P T_ij L_P^T (FP64 plans)."""
        _check(_load().ladder_plan_set_path(self._h, int(path)), "ladder_plan_set_path")

    def set_form(self, form: int):
        """Emulated ladder form: 0 plain, 1 symmetric/antisymmetric (see ladder_plan_set_form)."""
        _check(_load().ladder_plan_set_form(self._h, int(form)), "ladder_plan_set_form")

    def shard(self, rank: int, world: int):
        """Keep only the block pairs rank `rank` of `world` owns (see ladder_plan_shard)."""
        _check(_load().ladder_plan_shard(self._h, int(rank), int(world)), "ladder_plan_shard")

    def set_wait_limit(self, seconds: float):
        """Limit of the kernels' bounded waits (0 = the default 2 s); see ladder_plan_set_wait_limit."""
        _check(_load().ladder_plan_set_wait_limit(self._h, float(seconds)), "ladder_plan_set_wait_limit")

    def wait_limit(self) -> float:
        return float(_load().ladder_plan_get_wait_limit(self._h))

    def set_timing(self, enable: bool):
        _check(_load().ladder_plan_set_timing(self._h, int(bool(enable))), "ladder_plan_set_timing")

    def timing(self, kernel_class: int, reset: bool = False):
        """(summed ms, launches) of one kernel class since the last reset."""
        ms = ctypes.c_float()
        n = ctypes.c_int()
        _check(_load().ladder_plan_timing(self._h, int(kernel_class), ctypes.byref(ms), ctypes.byref(n), int(reset)),
               "ladder_plan_timing")
        return float(ms.value), int(n.value)

    def last_status(self, stream=None) -> int:
        return int(_load().ladder_last_status(self._h, _stream_handle(stream)))

    def close(self):
        if self._h:
            _load().ladder_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ladder_plan(no, nv, nchol, precision=LADDER_FP64, nslices=0, ws_budget_bytes=0, device=0) -> Plan:
    h = ctypes.c_void_p()
    _check(_load().ladder_plan(ctypes.byref(h), int(no), int(nv), int(nchol), int(precision), int(nslices),
                               int(ws_budget_bytes), int(device)), "ladder_plan")
    return Plan(h, no, nv, nchol, device)


def ladder_workspace_bytes(plan: Plan) -> int:
    return plan.workspace_bytes()


def ladder_apply(plan: Plan, L, t2, R, ws=None, stream=None):
    """R += ladder(L, t2) on the current (or given) stream; returns R."""
    if ws is None:
        ws = plan.workspace()
    _check(_load().ladder_apply(plan.handle, _dev_ptr(L, "L"), _dev_ptr(t2, "t2"), _dev_ptr(R, "R"),
                                ctypes.c_void_p(ws.data_ptr()), _stream_handle(stream)), "ladder_apply")
    return R


def _host_ptr(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host (CPU) tensor")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous float64")
    return ctypes.c_void_p(t.data_ptr())


def ladder_apply_host(plan: Plan, L, t2, R, stage=None, ws=None, stream=None):
    """R (host) = ladder(L, t2) from host tensors, through the plan's two device staging sets; the
    result is in R once the stream has been synchronised.  Returns R."""
    if stage is None:
        stage = plan.host_staging()
    if ws is None:
        ws = plan.workspace()
    _check(_load().ladder_apply_host(plan.handle, _host_ptr(L, "L"), _host_ptr(t2, "t2"), _host_ptr(R, "R"),
                                     ctypes.c_void_p(stage.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                     _stream_handle(stream)), "ladder_apply_host")
    return R


def ladder_energy(plan: Plan, t2, R, E_dev=None, stream=None):
    """E_L on the device (written to E_dev if given) and returned as a float when E_dev is None."""
    if E_dev is not None:
        _check(_load().ladder_energy(plan.handle, _dev_ptr(t2, "t2"), _dev_ptr(R, "R"), _dev_ptr(E_dev, "E_dev"),
                                     None, _stream_handle(stream)), "ladder_energy")
        return E_dev
    out = ctypes.c_double()
    _check(_load().ladder_energy(plan.handle, _dev_ptr(t2, "t2"), _dev_ptr(R, "R"), None, ctypes.byref(out),
                                 _stream_handle(stream)), "ladder_energy")
    return out.value


def ladder_plan_dry(no, nv, nchol, precision=LADDER_FP64, nslices=0, ws_budget_bytes=1 << 40, num_sms=152,
                    force_n_a=0, force_n_b=0, max_blocks=1 << 16):
    """Host-only planner run: returns dict(n_a, n_b, ws_bytes, blocks=[(a0, a1, b0, b1, npairs), ...])."""
    na, nb, nbp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ws = ctypes.c_size_t()
    buf = (ctypes.c_int * (5 * max_blocks))()
    _check(_load().ladder_plan_dry(int(no), int(nv), int(nchol), int(precision), int(nslices), int(ws_budget_bytes),
                                   int(num_sms), int(force_n_a), int(force_n_b), ctypes.byref(na), ctypes.byref(nb),
                                   ctypes.byref(ws), max_blocks, ctypes.byref(nbp), buf), "ladder_plan_dry")
    n = min(nbp.value, max_blocks)
    blocks = [tuple(buf[5 * k:5 * k + 5]) for k in range(n)]
    return {"n_a": na.value, "n_b": nb.value, "ws_bytes": ws.value, "n_block_pairs": nbp.value, "blocks": blocks}


def ladder_plan_shard_dry(no, nv, nchol, rank, world, precision=LADDER_FP64, nslices=0, ws_budget_bytes=1 << 40,
                          num_sms=152, max_blocks=1 << 16):
    """Host-only: the block pairs ladder_plan_shard keeps for rank `rank` of `world`, as
    dict(n_a, n_b, ws_bytes, blocks=[(a0, a1, b0, b1, npairs), ...])."""
    na, nb, nbp = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ws = ctypes.c_size_t()
    buf = (ctypes.c_int * (5 * max_blocks))()
    _check(_load().ladder_plan_shard_dry(int(no), int(nv), int(nchol), int(precision), int(nslices),
                                         int(ws_budget_bytes), int(num_sms), int(rank), int(world), ctypes.byref(na),
                                         ctypes.byref(nb), ctypes.byref(ws), max_blocks, ctypes.byref(nbp), buf),
           "ladder_plan_shard_dry")
    n = min(nbp.value, max_blocks)
    blocks = [tuple(buf[5 * k:5 * k + 5]) for k in range(n)]
    return {"n_a": na.value, "n_b": nb.value, "ws_bytes": ws.value, "n_block_pairs": nbp.value, "blocks": blocks}


def ladder_form_model(no, nv, nchol, nslices=0) -> int:
    """Form the emulated path's cost model picks for a shape (0 plain, 1 symmetric/antisymmetric)."""
    r = int(_load().ladder_form_model(int(no), int(nv), int(nchol), int(nslices)))
    if r < 0:
        raise LadderError(LADDER_ERR_ARG, "ladder_form_model")
    return r


def ladder_path_model(no, nv, nchol, precision=LADDER_FP64) -> int:
    """Evaluation order ladder_plan picks for a shape (0 rebuild, 1 factorised), host only."""
    r = int(_load().ladder_path_model(int(no), int(nv), int(nchol), int(precision)))
    if r < 0:
        raise LadderError(LADDER_ERR_ARG, "ladder_path_model")
    return r


def ladder_shard_blocks(npairs, world: int):
    """Owner rank of each block pair (pair counts `npairs`) when spread over `world` ranks."""
    n = len(npairs)
    arr = (ctypes.c_longlong * max(n, 1))(*map(int, npairs))
    owner = (ctypes.c_int * max(n, 1))()
    _check(_load().ladder_shard_blocks(n, arr, int(world), owner), "ladder_shard_blocks")
    return list(owner[:n])


def ladder_plan_shard(plan: Plan, rank: int, world: int) -> Plan:
    plan.shard(rank, world)
    return plan


def ladder_plan_batched(no, nv, nchol, precision=LADDER_EMU_BF16, nslices=0, ws_budget_bytes=0, device=0) -> Plan:
    n = len(no)
    arr = ctypes.c_int * n
    h = ctypes.c_void_p()
    _check(_load().ladder_plan_batched(ctypes.byref(h), n, arr(*map(int, no)), arr(*map(int, nv)),
                                       arr(*map(int, nchol)), int(precision), int(nslices), int(ws_budget_bytes),
                                       int(device)), "ladder_plan_batched")
    return Plan(h, device=device, batched_shapes=list(zip(no, nv, nchol)))


def ladder_apply_batched(plan: Plan, Ls, t2s, Rs, ws=None, stream=None):
    n = len(Ls)
    if not (len(t2s) == len(Rs) == n):
        raise ValueError("L, t2, R lists must have equal length")
    arr = ctypes.c_void_p * n
    a = arr(*[_dev_ptr(x, "L").value for x in Ls])
    b = arr(*[_dev_ptr(x, "t2").value for x in t2s])
    c = arr(*[_dev_ptr(x, "R").value for x in Rs])
    if ws is None:
        ws = plan.workspace()
    _check(_load().ladder_apply_batched(plan.handle, a, b, c, ctypes.c_void_p(ws.data_ptr()), _stream_handle(stream)),
           "ladder_apply_batched")
    return Rs


def ladder_batched_schedule(plan: Plan, schedule: int) -> int:
    """schedule > 0: that many worker streams; < 0: grouped, ws / |schedule| bytes per group.
    Returns the number of streams (> 0) or minus the number of groups."""
    out = ctypes.c_int()
    _check(_load().ladder_batched_schedule(plan.handle, int(schedule), ctypes.byref(out)), "ladder_batched_schedule")
    return out.value


def ladder_tune_batched(plan: Plan, Ls, t2s, Rs, ws=None, stream=None) -> int:
    """Time worker-stream and grouped schedules on these buffers (R receives every trial) and keep
    the fastest; returns the number of streams (> 0) or minus the number of groups (< 0)."""
    n = len(Ls)
    arr = ctypes.c_void_p * n
    a = arr(*[_dev_ptr(x, "L").value for x in Ls])
    b = arr(*[_dev_ptr(x, "t2").value for x in t2s])
    c = arr(*[_dev_ptr(x, "R").value for x in Rs])
    if ws is None:
        ws = plan.workspace()
    k = ctypes.c_int()
    _check(_load().ladder_tune_batched(plan.handle, a, b, c, ctypes.c_void_p(ws.data_ptr()), _stream_handle(stream),
                                       ctypes.byref(k)), "ladder_tune_batched")
    return k.value


def ladder_energy_noalloc(t2, R, E_dev, stream=None):
    """E_L into the device scalar E_dev without a plan and without any allocation.

    For callers that cannot allocate device memory (e.g. while a stream is being
    captured into a CUDA graph).  The scratch is a fixed 128 KiB device array inside
    the library, shared by every call: calls that may overlap on the GPU must be
    ordered.  The first call on a device should come before any stream capture."""
    no, _, nv, _ = t2.shape
    _check(_load().ladder_energy_noalloc(int(no), int(nv), _dev_ptr(t2, "t2"), _dev_ptr(R, "R"),
                                         _dev_ptr(E_dev, "E_dev"), _stream_handle(stream)), "ladder_energy_noalloc")
    return E_dev


def ladder_watchdog_selftest(limit_s=0.0, stream=None):
    """(status, waited_ms): status is LADDER_ERR_TIMEOUT when the bounded wait fired as designed
    (limit_s seconds of the GPU's global timer, 0 = the default 2 s)."""
    ms = ctypes.c_double()
    rc = _load().ladder_watchdog_selftest(float(limit_s), ctypes.byref(ms), _stream_handle(stream))
    return int(rc), ms.value


def ladder_last_status(plan: Plan, stream=None) -> int:
    return plan.last_status(stream)


def ladder_plan_destroy(plan: Plan):
    plan.close()


EXPORTED_SYMBOLS = [
    "ladder_plan", "ladder_plan_set_blocks", "ladder_workspace_bytes", "ladder_plan_describe", "ladder_apply",
    "ladder_energy", "ladder_plan_batched", "ladder_apply_batched", "ladder_last_status", "ladder_plan_destroy",
    "ladder_strerror", "ladder_flops", "ladder_plan_dry", "ladder_plan_set_timing", "ladder_plan_timing",
    "ladder_energy_noalloc", "ladder_tune_batched", "ladder_plan_shard", "ladder_shard_blocks",
    "ladder_watchdog_selftest", "ladder_batched_schedule", "ladder_plan_set_form", "ladder_plan_get_form",
    "ladder_form_model", "ladder_plan_set_wait_limit", "ladder_plan_get_wait_limit",
    "ladder_plan_shard_dry", "ladder_plan_set_path", "ladder_plan_get_path", "ladder_path_model",
    "ladder_plan_set_ladder_tile", "ladder_plan_get_ladder_tile", "ladder_plan_set_eri_chunk",
    "ladder_plan_eri_chunk", "ladder_plan_set_pbatch", "ladder_plan_get_pbatch", "ladder_apply_host",
    "ladder_host_staging_bytes",
]
