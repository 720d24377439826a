"""ctypes binding of libgcfvmc (the C ABI in include/gcfvmc.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  PyTorch provides device memory and the stream.  If the shared
library has not been built, loading fails with an error: there is no
fallback implementation.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgcfvmc.so")

GCF_OK, GCF_EINVAL, GCF_ENOMEM, GCF_ECUDA, GCF_EGAUSS, GCF_ENUMERIC, GCF_ETIMEOUT = range(7)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EGAUSS", "ENUMERIC", "ETIMEOUT"]
REAL, COMPLEX = 0, 1
FP64, FP32, TF32, BF16 = 0, 1, 2, 3
SR, TDVP_STAGE1, TDVP_STAGE2 = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32, "tf32": TF32, "bf16": BF16}


class GcfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"gcf status {STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class _Model(C.Structure):
    _fields_ = [("N", C.c_int), ("Lx", C.c_int), ("Ly", C.c_int), ("D", C.c_int), ("chi", C.c_int),
                ("has_matter", C.c_int), ("Q", C.POINTER(C.c_int32)), ("h", C.c_double),
                ("g", C.c_double), ("J", C.c_double), ("m", C.c_double), ("dtype", C.c_int),
                ("precision", C.c_int), ("trunc", C.c_int), ("recompute_env", C.c_int)]


class _Samples(C.Structure):
    _fields_ = [("log_abs", C.c_void_p), ("phase", C.c_void_p), ("e_loc", C.c_void_p),
                ("block_ids", C.c_void_p), ("O", C.c_void_p), ("accepted", C.c_void_p),
                ("proposed", C.c_void_p)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libgcfvmc.so (built by ``paper_2503_20566_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgcfvmc.so not built at {path}; run paper_2503_20566_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i, i64, d, u64 = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_uint64
    sigs = {
        "gcf_init_peps": (i, [C.POINTER(_Model), u64, vp, C.POINTER(vp)]),
        "gcf_destroy": (None, [vp]),
        "gcf_last_error": (C.c_char_p, [vp]),
        "gcf_num_params": (i64, [vp]),
        "gcf_config_len": (i, [vp]),
        "gcf_scalar_bytes": (i, [vp]),
        "gcf_launch_count": (i64, [vp]),
        "gcf_executor": (i, [vp]),
        "gcf_smem_level": (i, [vp]),
        "gcf_phase_timeouts": (i, [vp]),
        "gcf_svd_unconverged": (i, [vp]),
        "gcf_scratch_bytes_per_chain": (i64, [vp]),
        "gcf_checkpoint_interval": (i, [vp]),
        "gcf_tensor_core_form": (i, [vp]),
        "gcf_tensor_timeouts": (i, [vp]),
        "gcf_multi_chains_per_cta": (i, [vp]),
        "gcf_set_svd_sweeps": (i, [vp, i]),
        "gcf_autotune": (i, [vp, i, i, vp, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
        "gcf_set_tensors": (i, [vp, vp, C.c_size_t]),
        "gcf_get_tensors": (i, [vp, vp, C.c_size_t]),
        "gcf_init_configs": (i, [vp, i, vp, vp, vp]),
        "gcf_amplitude": (i, [vp, i, vp, vp, vp]),
        "gcf_local_energy": (i, [vp, i, vp, vp]),
        "gcf_log_grad": (i, [vp, i, vp, vp, vp]),
        "gcf_log_grad_vjp": (i, [vp, i, vp, vp, vp]),
        "gcf_sample_multi": (i, [C.POINTER(vp), i, C.POINTER(C.c_int), i, C.POINTER(C.c_uint64), C.POINTER(vp),
                                 C.POINTER(_Samples)]),
        "gcf_sample_batch": (i, [vp, i, i, u64, vp, C.POINTER(_Samples)]),
        "gcf_sample_batch_async": (i, [vp, i, i, u64, vp, C.POINTER(_Samples), vp]),
        "gcf_sr_step": (i, [vp, i, i, vp, vp, vp, d, d, i, d, i, d, C.POINTER(C.c_double)]),
        "gcf_vmc_step_host": (i, [vp, i, i, u64, vp, d, d, i, d, i, d, C.POINTER(C.c_double)]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names the binding expects the library to export."""
    return ["gcf_init_peps", "gcf_destroy", "gcf_last_error", "gcf_num_params", "gcf_config_len",
            "gcf_scalar_bytes", "gcf_launch_count", "gcf_executor", "gcf_smem_level", "gcf_phase_timeouts", "gcf_svd_unconverged", "gcf_set_svd_sweeps", "gcf_scratch_bytes_per_chain", "gcf_checkpoint_interval", "gcf_tensor_core_form", "gcf_tensor_timeouts", "gcf_multi_chains_per_cta", "gcf_autotune", "gcf_set_tensors", "gcf_get_tensors",
            "gcf_init_configs", "gcf_amplitude", "gcf_local_energy", "gcf_log_grad", "gcf_log_grad_vjp", "gcf_sample_multi",
            "gcf_sample_batch", "gcf_sample_batch_async", "gcf_sr_step", "gcf_vmc_step_host"]


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _need(cond, msg):
    if not cond:
        raise ValueError(msg)


def _check_device_buffers(bufs, device=None):
    """Buffers the library reads or writes through raw device pointers, as
    (tensor, dtype, min_numel, name): each must be a contiguous torch tensor of
    `dtype` with at least `min_numel` entries, on the GPU (on GPU `device`
    when given: the context's).  The C ABI cannot see a buffer's size or
    placement, so these are checked here, before any pointer is passed: first
    every shape and dtype, then the placement."""
    for t, dtype, min_numel, what in bufs:
        _need(hasattr(t, "data_ptr") and hasattr(t, "is_cuda"), f"{what} must be a torch tensor")
        _need(t.dtype == dtype, f"{what} must be {dtype}, got {t.dtype}")
        _need(t.numel() >= min_numel, f"{what} holds {t.numel()} entries, the call uses {min_numel}")
        _need(t.is_contiguous(), f"{what} must be contiguous")
    for t, _, _, what in bufs:
        _need(t.is_cuda, f"{what} must be on the GPU")
        _need(device is None or t.device.index == device,
              f"{what} is on cuda:{t.device.index}, the context lives on cuda:{device}")


def _check_configs(t, cfg_len, what, device=None):
    """In/out configurations: an int8 (n_chains, cfg_len) contiguous CUDA tensor."""
    import torch

    _need(hasattr(t, "dim") and t.dim() == 2 and t.shape[1] == cfg_len,
          f"{what}: configs must be (n_chains, {cfg_len}), got {tuple(getattr(t, 'shape', ()))}")
    _check_device_buffers([(t, torch.int8, t.shape[0] * cfg_len, f"{what}: configs")], device)


def _check_samples(out, n_chains, n_sweeps, n_s, D4, o_dtype, what, device=None):
    """Output buffers of a sampling call: every buffer present holds at least
    the entries the call writes, in the documented dtype."""
    import torch

    ns = n_chains * max(0, n_sweeps)
    need = {"log_abs": (torch.float64, ns), "phase": (torch.float64, ns), "e_loc": (torch.float64, 2 * ns),
            "block_ids": (torch.int32, ns * n_s), "O": (o_dtype, ns * n_s * D4),
            "accepted": (torch.int32, n_chains), "proposed": (torch.int32, n_chains)}
    _check_device_buffers([(out[key], dt, cnt, f"{what}: out[{key!r}]") for key, (dt, cnt) in need.items()
                           if out.get(key) is not None], device)


class Context:
    """One GCF-PEPS ansatz on one lattice (a ``gcf_ctx``)."""

    def __init__(self, N, Lx, Ly, D, chi, matter=False, Q=None, h=1.0, g=0.0, J=0.0, m=0.0,
                 complex_=False, precision="fp32", seed=0, stream=None, recompute_env=0):
        import torch

        _need(Q is None or np.asarray(Q).size == Lx * Ly, f"Q must hold Lx x Ly = {Lx * Ly} background charges")
        self._torch = torch
        self.lib = load_library()
        self.N, self.Lx, self.Ly, self.D, self.chi = N, Lx, Ly, D, chi
        self.Dk = D // N
        self.matter = bool(matter)
        self.complex = bool(complex_)
        self.precision = precision
        self.n_s = Lx * Ly
        self.n_plaq = (Lx - 1) * (Ly - 1)
        self.h, self.g, self.J, self.m = float(h), float(g), float(J), float(m)
        self.Q = None
        q = None
        if Q is not None:
            self._Q = np.ascontiguousarray(np.asarray(Q, dtype=np.int32).reshape(-1))
            self.Q = self._Q.copy()
            q = self._Q.ctypes.data_as(C.POINTER(C.c_int32))
        mdl = _Model(N, Lx, Ly, D, chi, int(matter), q, h, g, J, m, COMPLEX if complex_ else REAL,
                     PRECISIONS[precision], 0, int(recompute_env))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        # the library ties the context to the device current now; every call
        # must find it current again, and every buffer must live there
        self.device = torch.cuda.current_device()
        self._dev = torch.device("cuda", self.device)
        h_ctx = C.c_void_p()
        st = self.lib.gcf_init_peps(C.byref(mdl), C.c_uint64(seed), C.c_void_p(stream.cuda_stream),
                                    C.byref(h_ctx))
        if st != GCF_OK:
            raise GcfError(st, "gcf_init_peps failed")
        self.ctx = h_ctx
        self.n_params = int(self.lib.gcf_num_params(self.ctx))
        self.cfg_len = int(self.lib.gcf_config_len(self.ctx))
        self.scalar_bytes = int(self.lib.gcf_scalar_bytes(self.ctx))
        if precision == "fp64":
            self.o_dtype = torch.complex128 if complex_ else torch.float64
        else:
            self.o_dtype = torch.complex64 if complex_ else torch.float32

    # ---- lifecycle ------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.gcf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what, allow=()):
        if st != GCF_OK and st not in allow:
            msg = self.lib.gcf_last_error(self.ctx)
            raise GcfError(st, f"{what}: {msg.decode() if msg else ''}")
        return st

    @property
    def launch_count(self):
        return int(self.lib.gcf_launch_count(self.ctx))

    def autotune(self, configs, n_sweeps=1):
        """Time every kernel form on a copy of `configs` and keep the fastest.
        Returns the time (ms) of each form tried, in the library's order."""
        c = self._configs(configs)
        nf = C.c_int(16)
        ms = (C.c_double * 16)()
        self._check(self.lib.gcf_autotune(self.ctx, c.shape[0], int(n_sweeps), _ptr(c), ms, C.byref(nf)),
                    "autotune")
        return [float(ms[i]) for i in range(min(nf.value, 16))]

    @property
    def phase_timeouts(self):
        """Lockstep waits that ran out in the last synchronous launch."""
        return int(self.lib.gcf_phase_timeouts(self.ctx))

    @property
    def tensor_core_form(self):
        """True if the BF16 form's environment GEMMs run on tcgen05 tensor cores."""
        return bool(self.lib.gcf_tensor_core_form(self.ctx))

    @property
    def multi_chains_per_cta(self):
        """Chains per CTA of the last sample_multi launch with this context first."""
        return int(self.lib.gcf_multi_chains_per_cta(self.ctx))

    @property
    def tensor_timeouts(self):
        """Tensor-core waits that ran out in the last synchronous launch."""
        return int(self.lib.gcf_tensor_timeouts(self.ctx))

    @property
    def scratch_bytes_per_chain(self):
        """Device scratch of one chain slot (boundary-MPS store and buffers)."""
        return int(self.lib.gcf_scratch_bytes_per_chain(self.ctx))

    @property
    def checkpoint_interval(self):
        """K of the checkpointed boundary-MPS store, 0 when every MPS is kept."""
        return int(self.lib.gcf_checkpoint_interval(self.ctx))

    @property
    def svd_unconverged(self):
        """Truncated-bond SVDs that hit the sweep limit in the last synchronous launch."""
        return int(self.lib.gcf_svd_unconverged(self.ctx))

    def set_svd_sweeps(self, max_sweeps):
        """Sweep limit of the one-sided Jacobi SVD (default 40)."""
        self._check(self.lib.gcf_set_svd_sweeps(self.ctx, int(max_sweeps)), "set_svd_sweeps")

    @property
    def smem_level(self):
        return int(self.lib.gcf_smem_level(self.ctx))

    @property
    def kernel_name(self):
        """Name of the sampling / measurement kernel this context launches."""
        return {1: "gcf::vmc_kernel_grouped", 2: "gcf::vmc_kernel_grouped4"}.get(
            int(self.lib.gcf_executor(self.ctx)), "gcf::vmc_kernel")

    # ---- parameters -------------------------------------------------------
    def set_tensors(self, values):
        v = np.ascontiguousarray(np.asarray(values, dtype=np.complex128 if self.complex else np.float64))
        if v.shape != (self.n_params,):
            raise ValueError(f"expected {self.n_params} parameters")
        self._check(self.lib.gcf_set_tensors(self.ctx, v.ctypes.data_as(C.c_void_p), v.nbytes), "set_tensors")

    def get_tensors(self):
        v = np.zeros(self.n_params, dtype=np.complex128 if self.complex else np.float64)
        self._check(self.lib.gcf_get_tensors(self.ctx, v.ctypes.data_as(C.c_void_p), v.nbytes), "get_tensors")
        return v

    # ---- configurations ----------------------------------------------------
    def init_configs(self, n_chains, occupations=None, powers=None):
        torch = self._torch
        dev = self._dev
        occ = None if occupations is None else torch.as_tensor(occupations, dtype=torch.int8)
        pw = None if powers is None else torch.as_tensor(powers, dtype=torch.int8)
        _need(occ is None or occ.numel() == n_chains * self.n_s,
              f"init_configs: occupations must hold n_chains x {self.n_s} values")
        _need(pw is None or pw.numel() == n_chains * self.n_plaq,
              f"init_configs: powers must hold n_chains x {self.n_plaq} values")
        occ = None if occ is None else occ.to(dev).contiguous()
        pw = None if pw is None else pw.to(dev).contiguous()
        cfg = torch.empty((n_chains, self.cfg_len), dtype=torch.int8, device=dev)
        self._check(self.lib.gcf_init_configs(self.ctx, n_chains, _ptr(occ), _ptr(pw), _ptr(cfg)), "init_configs")
        return cfg

    def _configs(self, configs):
        torch = self._torch
        c = torch.as_tensor(configs, dtype=torch.int8)
        if c.dim() == 1:
            c = c.unsqueeze(0)
        _need(c.dim() == 2 and c.shape[1] == self.cfg_len,
              f"configs must be (n, {self.cfg_len}), got {tuple(c.shape)}")
        return c.to(self._dev).contiguous()

    # ---- fixed-configuration evaluations ---------------------------------------
    def amplitude(self, configs):
        torch = self._torch
        c = self._configs(configs)
        n = c.shape[0]
        la = torch.empty(n, dtype=torch.float64, device=self._dev)
        ph = torch.empty(n, dtype=torch.float64, device=self._dev)
        self._check(self.lib.gcf_amplitude(self.ctx, n, _ptr(c), _ptr(la), _ptr(ph)), "amplitude")
        return la, ph

    def local_energy(self, configs):
        torch = self._torch
        c = self._configs(configs)
        n = c.shape[0]
        e = torch.empty(2 * n, dtype=torch.float64, device=self._dev)
        self._check(self.lib.gcf_local_energy(self.ctx, n, _ptr(c), _ptr(e)), "local_energy")
        return torch.view_as_complex(e.view(n, 2))

    def log_grad(self, configs):
        torch = self._torch
        c = self._configs(configs)
        n = c.shape[0]
        D4 = self.Dk ** 4
        bid = torch.empty((n, self.n_s), dtype=torch.int32, device=self._dev)
        O = torch.zeros((n, self.n_s, D4), dtype=self.o_dtype, device=self._dev)
        self._check(self.lib.gcf_log_grad(self.ctx, n, _ptr(c), _ptr(bid), _ptr(O)), "log_grad")
        return bid, O

    def log_grad_vjp(self, configs, weights):
        """sum_s w_s d ln psi(s) / d theta as a device tensor of n_params
        (complex128 for complex tensors)."""
        torch = self._torch
        c = self._configs(configs)
        n = c.shape[0]
        if self.complex:
            w = torch.view_as_real(torch.as_tensor(weights, dtype=torch.complex128).to(self._dev).contiguous())
            g = torch.empty((self.n_params, 2), dtype=torch.float64, device=self._dev)
        else:
            w = torch.as_tensor(weights, dtype=torch.float64).to(self._dev).contiguous()
            g = torch.empty(self.n_params, dtype=torch.float64, device=self._dev)
        if w.shape[0] != n:
            raise ValueError(f"expected {n} weights")
        self._check(self.lib.gcf_log_grad_vjp(self.ctx, n, _ptr(c), _ptr(w), _ptr(g)), "log_grad_vjp")
        return torch.view_as_complex(g) if self.complex else g

    # ---- sampling and SR ---------------------------------------------------------
    def alloc_samples(self, n_chains, n_sweeps, grad=True):
        torch = self._torch
        ns = n_chains * n_sweeps
        out = {
            "log_abs": torch.empty(ns, dtype=torch.float64, device=self._dev),
            "phase": torch.empty(ns, dtype=torch.float64, device=self._dev),
            "e_loc": torch.empty(2 * ns, dtype=torch.float64, device=self._dev),
            "accepted": torch.zeros(n_chains, dtype=torch.int32, device=self._dev),
            "proposed": torch.zeros(n_chains, dtype=torch.int32, device=self._dev),
        }
        if grad:
            out["block_ids"] = torch.empty((ns, self.n_s), dtype=torch.int32, device=self._dev)
            out["O"] = torch.zeros((ns, self.n_s, self.Dk ** 4), dtype=self.o_dtype, device=self._dev)
        return out

    def sample_batch(self, configs, n_sweeps, seed, out=None, grad=True):
        """configs: device int8 tensor (n_chains, cfg_len), updated in place."""
        _check_configs(configs, self.cfg_len, "sample_batch", self.device)
        n = configs.shape[0]
        if out is None:
            out = self.alloc_samples(n, n_sweeps, grad)
        _check_samples(out, n, n_sweeps, self.n_s, self.Dk ** 4, self.o_dtype, "sample_batch", self.device)
        s = _Samples(*[C.c_void_p(out[k].data_ptr()) if k in out else None
                       for k in ("log_abs", "phase", "e_loc", "block_ids", "O", "accepted", "proposed")])
        self._check(self.lib.gcf_sample_batch(self.ctx, n, n_sweeps, C.c_uint64(seed), _ptr(configs),
                                              C.byref(s)), "sample_batch")
        return out

    def sample_batch_async(self, configs, n_sweeps, seed, out, stream=None):
        """Enqueue sample_batch on `stream` (a torch.cuda.Stream; default the
        context's) without synchronising or allocating: the launch can be
        recorded in a CUDA graph.  Call sample_batch with at least as many
        chains once before (it sizes the scratch)."""
        _check_configs(configs, self.cfg_len, "sample_batch_async", self.device)
        n = configs.shape[0]
        _check_samples(out, n, n_sweeps, self.n_s, self.Dk ** 4, self.o_dtype, "sample_batch_async", self.device)
        h = None if stream is None else C.c_void_p(stream.cuda_stream)
        s = _samples_struct(out)
        self._check(self.lib.gcf_sample_batch_async(self.ctx, n, n_sweeps, C.c_uint64(seed), _ptr(configs),
                                                    C.byref(s), h), "sample_batch_async")
        return out

    def sr_step(self, samples, n_chains, diag_shift=1e-4, lr=0.01, mode=SR, dt=0.0, max_iter=100,
                tol=1e-10):
        torch = self._torch
        ns = samples["e_loc"].shape[0] // 2
        _check_device_buffers([(samples["e_loc"], torch.float64, 2 * ns, "sr_step: samples['e_loc']"),
                               (samples["block_ids"], torch.int32, ns * self.n_s, "sr_step: samples['block_ids']"),
                               (samples["O"], self.o_dtype, ns * self.n_s * self.Dk ** 4, "sr_step: samples['O']")],
                              self.device)
        stats = (C.c_double * 8)()
        st = self.lib.gcf_sr_step(self.ctx, ns, n_chains, _ptr(samples["e_loc"]), _ptr(samples["block_ids"]),
                                  _ptr(samples["O"]), diag_shift, lr, mode, dt, max_iter, tol, stats)
        self._check(st, "sr_step", allow=(GCF_ETIMEOUT,))
        return list(stats)

    def vmc_step_host(self, host_configs, n_sweeps, seed, diag_shift=1e-4, lr=0.01, mode=SR, dt=0.0,
                      max_iter=100, tol=1e-10):
        """One VMC iteration from host memory (configs: numpy int8, in/out)."""
        _need(isinstance(host_configs, np.ndarray) and host_configs.dtype == np.int8 and
              host_configs.flags["C_CONTIGUOUS"] and host_configs.flags["WRITEABLE"],
              "vmc_step_host: configs must be a writeable, contiguous numpy int8 array")
        _need(host_configs.ndim == 2 and host_configs.shape[1] == self.cfg_len,
              f"vmc_step_host: configs must be (n_chains, {self.cfg_len}), got {host_configs.shape}")
        n = host_configs.shape[0]
        stats = (C.c_double * 8)()
        st = self.lib.gcf_vmc_step_host(self.ctx, n, n_sweeps, C.c_uint64(seed),
                                        host_configs.ctypes.data_as(C.c_void_p), diag_shift, lr, mode, dt,
                                        max_iter, tol, stats)
        self._check(st, "vmc_step_host", allow=(GCF_ETIMEOUT,))
        return list(stats)


def _samples_struct(out):
    return _Samples(*[C.c_void_p(out[k].data_ptr()) if k in out else None
                      for k in ("log_abs", "phase", "e_loc", "block_ids", "O", "accepted", "proposed")])


def sample_multi(contexts, configs, n_sweeps, seeds, outs=None, grad=True):
    """gcf_sample_multi: the chains of several contexts (lattices of different
    sizes) in one launch.  configs[i]: device int8 (n_chains_i, cfg_len_i),
    updated in place; seeds[i]: the seed context i would get from
    sample_batch.  Returns the per-context output dicts."""
    n = len(contexts)
    if not (len(configs) == len(seeds) == n) or n == 0:
        raise ValueError("one configs tensor and one seed per context")
    for i, (ctx, c) in enumerate(zip(contexts, configs)):
        _check_configs(c, ctx.cfg_len, f"sample_multi[{i}]", ctx.device)
    if outs is None:
        outs = [ctx.alloc_samples(c.shape[0], n_sweeps, grad) for ctx, c in zip(contexts, configs)]
    _need(len(outs) == n, "one output dict per context")
    for i, (ctx, c, o) in enumerate(zip(contexts, configs, outs)):
        _check_samples(o, c.shape[0], n_sweeps, ctx.n_s, ctx.Dk ** 4, ctx.o_dtype, f"sample_multi[{i}]", ctx.device)
    lib = contexts[0].lib
    ctxs = (C.c_void_p * n)(*[ctx.ctx for ctx in contexts])
    nch = (C.c_int * n)(*[int(c.shape[0]) for c in configs])
    sds = (C.c_uint64 * n)(*[int(v) for v in seeds])
    cfg = (C.c_void_p * n)(*[c.data_ptr() for c in configs])
    smp = (_Samples * n)(*[_samples_struct(o) for o in outs])
    contexts[0]._check(lib.gcf_sample_multi(ctxs, n, nch, int(n_sweeps), sds, cfg, smp), "sample_multi")
    return outs
