"""Python API over the C ABI: a PPPM plan operating on torch device tensors.

PyTorch provides device memory and streams only; the arithmetic runs in the
CUDA library (``libpppm.so``).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Plan:
    """PPPM (Poisson-ik) for the Gaussian-charge energy E_Gt of DPLR in one
    orthorhombic box.

    box: 3 edge lengths (Angstrom); mesh: 3 mesh sizes (2^a 3^b 5^c);
    order: B-spline order p; beta: splitting parameter (1/Angstrom);
    precision: "fp32" or "fp64".
    """

    def __init__(self, box, mesh, order: int = 5, beta: float = 0.4, precision: str = "fp32",
                 prefactor: float = 1.0, alias: int = 2, tile: int = 0):
        L = N.lib()
        self._lib = L
        self.box = tuple(float(b) for b in np.broadcast_to(np.asarray(box, float), (3,)))
        self.mesh = tuple(int(m) for m in np.broadcast_to(np.asarray(mesh), (3,)))
        self.order = int(order)
        self.beta = float(beta)
        self.precision = precision
        prec = {"fp32": N.PPPM_FP32, "fp64": N.PPPM_FP64}[precision]
        self.real_dtype = torch.float32 if prec == N.PPPM_FP32 else torch.float64
        b = (ctypes.c_double * 3)(*self.box)
        m = (ctypes.c_int * 3)(*self.mesh)
        h = ctypes.c_void_p()
        N.check(L.pppm_create(b, m, self.order, self.beta, prec, ctypes.byref(h)), "pppm_create")
        self._h = h
        opt = N.Options()
        N.check(L.pppm_default_options(ctypes.byref(opt)))
        opt.prefactor, opt.alias, opt.tile = float(prefactor), int(alias), int(tile)
        N.check(L.pppm_set_options(self._h, ctypes.byref(opt)), "pppm_set_options")

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pppm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_options(self, prefactor=None, alias=None, tile=None):
        opt = N.Options()
        N.check(self._lib.pppm_get_options(self._h, ctypes.byref(opt)))
        if prefactor is not None:
            opt.prefactor = float(prefactor)
        if alias is not None:
            opt.alias = int(alias)
        if tile is not None:
            opt.tile = int(tile)
        N.check(self._lib.pppm_set_options(self._h, ctypes.byref(opt)), "pppm_set_options")

    def set_dependent_launch(self, on: bool = True):
        """Programmatic dependent launch between the kernels of an evaluation
        (default on; off may overlap better with concurrent work)."""
        N.check(self._lib.pppm_set_dependent_launch(self._h, int(bool(on))), "pppm_set_dependent_launch")

    def set_wait_limit(self, spins: int):
        """Polls of the gather's bounded wait for its tile copies (0: every
        first wait runs out, the call reports PPPM_ERR_TIMEOUT)."""
        N.check(self._lib.pppm_set_wait_limit(self._h, int(spins)), "pppm_set_wait_limit")

    def reserve(self, n: int):
        N.check(self._lib.pppm_reserve(self._h, int(n)), "pppm_reserve")

    def profile(self, on: bool = True):
        N.check(self._lib.pppm_profile_enable(self._h, int(bool(on))))

    def profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} since the last read (synchronizes)."""
        ms = (ctypes.c_double * 32)()
        calls = (ctypes.c_int64 * 32)()
        k = self._lib.pppm_profile_read(self._h, ms, calls, 32)
        if k < 0:
            N.check(k, "pppm_profile_read")
        return {self._lib.pppm_profile_name(i).decode(): (ms[i], calls[i]) for i in range(k)}

    def status(self) -> int:
        return self._lib.pppm_status(self._h)

    # ------------------------------------------------------------ compute
    @staticmethod
    def _check_sites(pos, q):
        if pos.dim() != 2 or pos.shape[1] != 3 or q.dim() != 1 or q.shape[0] != pos.shape[0]:
            raise ValueError("pos must be (n, 3) and q (n,)")
        if not (pos.is_cuda and q.is_cuda and pos.is_contiguous() and q.is_contiguous()):
            raise ValueError("pos and q must be contiguous CUDA tensors")
        if pos.dtype != q.dtype or pos.dtype not in (torch.float32, torch.float64):
            raise ValueError("pos and q must both be float32 or both float64")

    def compute(self, pos: torch.Tensor, q: torch.Tensor, out=None, stream=None):
        """Energy (1,), forces (n, 3) and virial (6,) as device tensors.
        float32 inputs use pppm_compute_f32, float64 pppm_compute."""
        self._check_sites(pos, q)
        n = pos.shape[0]
        if out is None:
            energy = torch.empty(1, dtype=torch.float64, device=pos.device)
            forces = torch.empty((n, 3), dtype=pos.dtype, device=pos.device)
            virial = torch.empty(6, dtype=torch.float64, device=pos.device)
        else:
            energy, forces, virial = out
        fn = self._lib.pppm_compute_f32 if pos.dtype == torch.float32 else self._lib.pppm_compute
        N.check(fn(self._h, _stream(stream), _ptr(pos), _ptr(q), n, _ptr(energy), _ptr(forces), _ptr(virial)),
                "pppm_compute")
        return energy, forces, virial

    def compute_host(self, pos: np.ndarray, q: np.ndarray, out=None):
        """The same evaluation from host numpy arrays (copies inside the call).
        out = (energy (1,), forces (n, 3), virial (6,)) host arrays to fill
        (pinned memory makes the device-to-host copies direct)."""
        pos = np.ascontiguousarray(pos)
        q = np.ascontiguousarray(q, dtype=pos.dtype)
        n = pos.shape[0]
        if out is None:
            energy = np.zeros(1)
            virial = np.zeros(6)
            forces = np.zeros((n, 3), dtype=pos.dtype)
        else:
            energy, forces, virial = out
            if (energy.dtype != np.float64 or virial.dtype != np.float64 or forces.dtype != pos.dtype
                    or forces.shape != (n, 3) or not forces.flags.c_contiguous):
                raise ValueError("out must be (float64 (1,), (n, 3) of the site dtype, float64 (6,))")
        fn = self._lib.pppm_compute_host_f32 if pos.dtype == np.float32 else self._lib.pppm_compute_host
        rc = fn(self._h, pos.ctypes.data, q.ctypes.data, n, energy.ctypes.data, forces.ctypes.data,
                virial.ctypes.data)
        N.check(rc, "pppm_compute_host")
        return float(energy[0]), forces, virial

    def graph(self, pos: torch.Tensor, q: torch.Tensor, out=None, stream=None) -> "StepGraph":
        """Capture one force evaluation as a CUDA graph (see StepGraph)."""
        return StepGraph(self, pos, q, out=out, stream=stream)

    # ------------------------------------------------------------ stages
    def spread(self, pos: torch.Tensor, q: torch.Tensor, stream=None) -> torch.Tensor:
        """Charge density on the mesh (plan precision), from float64 sites."""
        pos = pos.to(torch.float64).contiguous()
        q = q.to(torch.float64).contiguous()
        rho = torch.empty(self.mesh, dtype=self.real_dtype, device=pos.device)
        N.check(self._lib.pppm_spread(self._h, _stream(stream), _ptr(pos), _ptr(q), pos.shape[0], _ptr(rho)),
                "pppm_spread")
        return rho

    def fft_r2c(self, real: torch.Tensor, stream=None) -> torch.Tensor:
        assert real.dtype == self.real_dtype and tuple(real.shape) == self.mesh and real.is_contiguous()
        hz = self.mesh[2] // 2 + 1
        out = torch.empty((self.mesh[0], self.mesh[1], hz, 2), dtype=self.real_dtype, device=real.device)
        N.check(self._lib.pppm_fft_r2c(self._h, _stream(stream), _ptr(real), _ptr(out)), "pppm_fft_r2c")
        return torch.view_as_complex(out)

    def fft_c2r(self, spec: torch.Tensor, stream=None) -> torch.Tensor:
        spec = torch.view_as_real(spec.contiguous()).contiguous()
        assert spec.dtype == self.real_dtype
        out = torch.empty(self.mesh, dtype=self.real_dtype, device=spec.device)
        N.check(self._lib.pppm_fft_c2r(self._h, _stream(stream), _ptr(spec), _ptr(out)), "pppm_fft_c2r")
        return out

    def influence(self, device="cuda") -> torch.Tensor:
        hz = self.mesh[2] // 2 + 1
        G = torch.empty((self.mesh[0], self.mesh[1], hz), dtype=torch.float64, device=device)
        N.check(self._lib.pppm_influence(self._h, _ptr(G)), "pppm_influence")
        return G

    def fields(self, pos: torch.Tensor, q: torch.Tensor, stream=None) -> torch.Tensor:
        pos = pos.to(torch.float64).contiguous()
        q = q.to(torch.float64).contiguous()
        f = torch.empty((3,) + self.mesh, dtype=self.real_dtype, device=pos.device)
        N.check(self._lib.pppm_fields(self._h, _stream(stream), _ptr(pos), _ptr(q), pos.shape[0], _ptr(f)),
                "pppm_fields")
        return f


class StepGraph:
    """One captured force evaluation of a plan, replayed with launch().

    The outputs (energy, forces, virial: ``self.out``), the site count and the
    plan's options are fixed at capture; launch() may pass new position and
    charge tensors of the same shape and dtype.  The capture stream must not be
    the legacy default stream; by default a dedicated stream is used."""

    def __init__(self, plan: Plan, pos, q, out=None, stream=None):
        Plan._check_sites(pos, q)
        L = N.lib()
        self._lib = L
        self.plan = plan
        n = pos.shape[0]
        if out is None:
            out = (torch.empty(1, dtype=torch.float64, device=pos.device),
                   torch.empty((n, 3), dtype=pos.dtype, device=pos.device),
                   torch.empty(6, dtype=torch.float64, device=pos.device))
        self.out = out
        self.dtype = pos.dtype
        self.shape = tuple(pos.shape)
        if stream is None:
            stream = torch.cuda.Stream(device=pos.device)
        self.stream = stream
        # the capture's warm-up call uses the plan's workspace: order it after
        # the caller's work on the current stream
        stream.wait_stream(torch.cuda.current_stream(pos.device))
        h = ctypes.c_void_p()
        fn = L.pppm_graph_create_f32 if pos.dtype == torch.float32 else L.pppm_graph_create
        N.check(fn(plan.handle, _stream(stream), _ptr(pos), _ptr(q), n, _ptr(out[0]), _ptr(out[1]), _ptr(out[2]),
                   ctypes.byref(h)), "pppm_graph_create")
        self._h = h
        stream.synchronize()  # the capture's warm-up call shares the plan's workspace with later launches
        self._refs = (pos, q)

    def launch(self, pos=None, q=None, stream=None):
        """Replay on `stream` (default: the capture stream) with new sites (or
        the previous ones); returns the output tensors."""
        for t in (pos, q):
            if t is not None and (t.dtype != self.dtype or not t.is_cuda or not t.is_contiguous()):
                raise ValueError("sites must be contiguous CUDA tensors of the captured dtype")
        if pos is not None and tuple(pos.shape) != self.shape:
            raise ValueError("the site count is fixed at capture")
        fn = self._lib.pppm_graph_launch_f32 if self.dtype == torch.float32 else self._lib.pppm_graph_launch
        N.check(fn(self._h, _stream(stream if stream is not None else self.stream), _ptr(pos), _ptr(q)),
                "pppm_graph_launch")
        self._refs = (pos if pos is not None else self._refs[0], q if q is not None else self._refs[1])
        return self.out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pppm_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchPlan:
    """Many independent boxes in one persistent launch (FP32).

    boxes: (nbox, 3) edge lengths; meshes: (nbox, 3) or None for about 1.2 A
    spacing rounded up to 2^a 3^b 5^c; order 3, 5 or 7.
    """

    def __init__(self, boxes, meshes=None, order: int = 5, beta: float = 0.4, prefactor: float = 1.0,
                 tile: int = 0, spin_limit: int = 1 << 24):
        L = N.lib()
        self._lib = L
        boxes = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 3)
        self.nbox = boxes.shape[0]
        h = ctypes.c_void_p()
        mp = None
        if meshes is not None:
            m = np.ascontiguousarray(meshes, dtype=np.int32).reshape(-1, 3)
            mp = m.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        N.check(L.pppm_batch_create(self.nbox, boxes.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), mp,
                                    int(order), float(beta), ctypes.byref(h)), "pppm_batch_create")
        self._h = h
        self.boxes = boxes
        self.set(prefactor=prefactor, tile=tile, spin_limit=spin_limit)

    def set(self, prefactor: float = 1.0, tile: int = 0, spin_limit: int = 1 << 24):
        N.check(self._lib.pppm_batch_set(self._h, float(prefactor), int(tile), int(spin_limit)), "pppm_batch_set")

    def set_launch(self, form: str):
        """The launch form: "persistent" (one persistent kernel), "staged"
        (one kernel per stage over all boxes) or "auto" (the autotuner keeps
        the faster; default)."""
        mode = {"persistent": N.PPPM_BATCH_PERSISTENT, "staged": N.PPPM_BATCH_STAGED, "auto": N.PPPM_BATCH_AUTO}[form]
        N.check(self._lib.pppm_batch_set_launch(self._h, mode), "pppm_batch_set_launch")

    @property
    def launch(self) -> str:
        m = self._lib.pppm_batch_launch(self._h)
        return {N.PPPM_BATCH_PERSISTENT: "persistent", N.PPPM_BATCH_STAGED: "staged", N.PPPM_BATCH_AUTO: "auto"}[m]

    def set_wait_probe(self, on: bool):
        """When on, the first box's scan waits for one binning item more
        than exist, so that bounded wait must run out."""
        N.check(self._lib.pppm_batch_set_wait_probe(self._h, int(bool(on))), "pppm_batch_set_wait_probe")

    def set_dft(self, max_len: int):
        """Lines of length <= max_len (0..18, 0 = off) take the tensor-core
        DFT instead of the FFT."""
        N.check(self._lib.pppm_batch_set_dft(self._h, int(max_len)), "pppm_batch_set_dft")

    def set_quantized(self, group: int, scale: float = 1e7):
        """group > 0: lines of length <= 18 divisible by group take the
        int32-quantised per-node DFT at `scale` (an accuracy ablation; order
        5 only); 0 = off."""
        N.check(self._lib.pppm_batch_set_quantized(self._h, int(group), float(scale)), "pppm_batch_set_quantized")

    @property
    def meshes(self) -> np.ndarray:
        m = np.zeros((self.nbox, 3), dtype=np.int32)
        N.check(self._lib.pppm_batch_meshes(self._h, m.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return m

    @property
    def tile(self) -> int:
        return self._lib.pppm_batch_tile(self._h)

    def status(self) -> int:
        return self._lib.pppm_batch_status(self._h)

    def compute(self, pos: torch.Tensor, q: torch.Tensor, offsets: torch.Tensor, out=None, stream=None):
        """Energies (nbox,), forces (n, 3) and virials (nbox, 6) for the
        concatenated float32 sites; box b owns offsets[b]:offsets[b+1]."""
        if pos.dtype != torch.float32 or q.dtype != torch.float32 or offsets.dtype != torch.int64:
            raise ValueError("pos and q must be float32, offsets int64")
        if not (pos.is_cuda and q.is_cuda and offsets.is_cuda):
            raise ValueError("tensors must be on the GPU")
        n = pos.shape[0]
        dev = pos.device
        if out is None:
            energies = torch.empty(self.nbox, dtype=torch.float64, device=dev)
            forces = torch.empty((n, 3), dtype=torch.float32, device=dev)
            virials = torch.empty((self.nbox, 6), dtype=torch.float64, device=dev)
        else:
            energies, forces, virials = out
        N.check(self._lib.pppm_compute_batched(self._h, _stream(stream), _ptr(pos), _ptr(q), _ptr(offsets),
                                               _ptr(energies), _ptr(forces), _ptr(virials)), "pppm_compute_batched")
        return energies, forces, virials

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pppm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Corrector:
    """Learned correction of a coarse-mesh FP32 PPPM (see include/pppm.h,
    pppm_corr_*): per-site features of the coarse mesh potential go through an
    n_in-64-64-3 tanh network with BF16 weights; its output, times q_i s_out,
    is added to the coarse forces.  Training runs on the GPU (forward,
    backward and Adam in the library's own kernels) against fine-mesh forces.

    features: "cell" (48 inputs: 27 potential samples, site type, offset
    inside the mesh cell) or "stated" (32 inputs: the samples and the type).
    """

    WIDTH = {"cell": 48, "stated": 32}
    N_IN = 48  # width of the default ("cell") set

    def __init__(self, coarse: Plan, params=None, s_in: float = 1.0, s_out: float = 1.0, features: str = "cell"):
        if coarse.precision != "fp32":
            raise ValueError("the correction runs on an FP32 coarse plan")
        L = N.lib()
        self._lib = L
        self.coarse = coarse  # keeps the borrowed plan alive
        h = ctypes.c_void_p()
        kind = {"cell": N.PPPM_CORR_CELL, "stated": N.PPPM_CORR_STATED}[features]
        N.check(L.pppm_corr_create_features(coarse.handle, kind, ctypes.byref(h)), "pppm_corr_create_features")
        self._h = h
        self.features_kind = features
        self.n_in = int(L.pppm_corr_feature_width(h))
        self.nparams = int(L.pppm_corr_param_count(h))
        self.forward_kind = "mma_sync"
        if params is not None:
            self.set_weights(params, s_in, s_out)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pppm_corr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_forward(self, kind: str):
        """Kernel of the network forward: "mma_sync" (default; warp-level,
        the layers chained in registers) or "tcgen05" (tensor-memory
        accumulators, 128 sites a tile)."""
        k = {"tcgen05": N.PPPM_FORWARD_TCGEN05, "mma_sync": N.PPPM_FORWARD_MMA_SYNC}[kind]
        N.check(self._lib.pppm_corr_set_forward(self._h, k), "pppm_corr_set_forward")
        self.forward_kind = kind

    def set_wait_limit(self, spins: int):
        """Polls of the tcgen05 forward's wait for each MMA completion (0: every
        first wait runs out, to test the timeout path)."""
        N.check(self._lib.pppm_corr_set_wait_limit(self._h, int(spins)), "pppm_corr_set_wait_limit")

    # ------------------------------------------------------------ parameters
    def set_weights(self, params, s_in: float, s_out: float):
        p = np.ascontiguousarray(params, dtype=np.float32).ravel()
        if p.size != self.nparams:
            raise ValueError(f"expected {self.nparams} parameters, got {p.size}")
        N.check(self._lib.pppm_corr_set_weights(self._h, p.ctypes.data, float(s_in), float(s_out)),
                "pppm_corr_set_weights")

    def get_weights(self):
        p = np.empty(self.nparams, dtype=np.float32)
        si, so = ctypes.c_double(), ctypes.c_double()
        N.check(self._lib.pppm_corr_get_weights(self._h, p.ctypes.data, ctypes.byref(si), ctypes.byref(so)),
                "pppm_corr_get_weights")
        return p, si.value, so.value

    @property
    def scales(self):
        si, so = ctypes.c_double(), ctypes.c_double()
        N.check(self._lib.pppm_corr_get_scales(self._h, ctypes.byref(si), ctypes.byref(so)))
        return si.value, so.value

    def save(self, path: str):
        N.check(self._lib.pppm_corr_save(self._h, str(path).encode()), "pppm_corr_save")

    def load(self, path: str):
        N.check(self._lib.pppm_corr_load(self._h, str(path).encode()), "pppm_corr_load")

    # ------------------------------------------------------------ checks
    @staticmethod
    def _sites(pos, q, types):
        Plan._check_sites(pos, q)
        if pos.dtype != torch.float32:
            raise ValueError("the correction takes float32 sites")
        if types.dtype != torch.int8 or types.shape != q.shape or not (types.is_cuda and types.is_contiguous()):
            raise ValueError("types must be a contiguous int8 CUDA tensor of shape (n,)")

    def _check_table(self, feat, target, idx):
        if feat.dtype != torch.bfloat16 or feat.dim() != 2 or feat.shape[1] != self.n_in or not feat.is_contiguous():
            raise ValueError("feat must be a contiguous (n, 32) bfloat16 tensor")
        if target.dtype != torch.float32 or tuple(target.shape) != (feat.shape[0], 3) or not target.is_contiguous():
            raise ValueError("target must be a contiguous (n, 3) float32 tensor")
        if idx is not None and (idx.dtype != torch.int32 or idx.dim() != 1 or not idx.is_contiguous()):
            raise ValueError("idx must be a contiguous 1-D int32 tensor")

    # ------------------------------------------------------------ evaluation
    def features(self, pos, q, types, feat=None, forces=None, stream=None):
        """Coarse forces (n, 3) and features (n, 32) bf16."""
        self._sites(pos, q, types)
        n = pos.shape[0]
        if feat is None:
            feat = torch.empty((n, self.n_in), dtype=torch.bfloat16, device=pos.device)
        if forces is None:
            forces = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
        N.check(self._lib.pppm_corr_features(self._h, _stream(stream), _ptr(pos), _ptr(q), _ptr(types), n,
                                             _ptr(feat), _ptr(forces)), "pppm_corr_features")
        return feat, forces

    def forward(self, feat, out=None, stream=None):
        n = feat.shape[0]
        assert feat.dtype == torch.bfloat16 and feat.is_contiguous() and feat.shape[1] == self.n_in
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float32, device=feat.device)
        N.check(self._lib.pppm_corr_forward(self._h, _stream(stream), _ptr(feat), n, _ptr(out)),
                "pppm_corr_forward")
        return out

    def apply(self, pos, q, types, out=None, stream=None):
        """Corrected PPPM: energy (1,), forces (n, 3), virial (6,) (energy and
        virial are the coarse mesh's)."""
        self._sites(pos, q, types)
        n = pos.shape[0]
        if out is None:
            energy = torch.empty(1, dtype=torch.float64, device=pos.device)
            forces = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
            virial = torch.empty(6, dtype=torch.float64, device=pos.device)
        else:
            energy, forces, virial = out
        N.check(self._lib.pppm_corr_apply(self._h, _stream(stream), _ptr(pos), _ptr(q), _ptr(types), n,
                                          _ptr(energy), _ptr(forces), _ptr(virial)), "pppm_corr_apply")
        return energy, forces, virial

    # ------------------------------------------------------------ training
    def calibrate(self, pos, q, types, f_fine, stream=None):
        self._sites(pos, q, types)
        N.check(self._lib.pppm_corr_calibrate(self._h, _stream(stream), _ptr(pos), _ptr(q), _ptr(types),
                                              pos.shape[0], _ptr(f_fine.contiguous())), "pppm_corr_calibrate")
        return self.scales

    def targets(self, f_fine, f_coarse, q, out=None, stream=None):
        n = q.shape[0]
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float32, device=q.device)
        N.check(self._lib.pppm_corr_targets(self._h, _stream(stream), _ptr(f_fine), _ptr(f_coarse), _ptr(q), n,
                                            _ptr(out)), "pppm_corr_targets")
        return out

    def grad(self, feat, target, idx=None, nb=None, stream=None):
        """Loss (device scalar) and gradient (device, nparams) over rows idx
        (int32 device tensor) or the first nb rows."""
        self._check_table(feat, target, idx)
        nb = int(idx.shape[0]) if idx is not None else int(nb if nb is not None else feat.shape[0])
        g = torch.empty(self.nparams, dtype=torch.float32, device=feat.device)
        loss = torch.empty(1, dtype=torch.float32, device=feat.device)
        N.check(self._lib.pppm_corr_grad(self._h, _stream(stream), _ptr(feat), _ptr(target), feat.shape[0],
                                         _ptr(idx), nb, _ptr(g), _ptr(loss)), "pppm_corr_grad")
        return loss, g

    def train_step(self, feat, target, idx, lr: float, loss=None, stream=None):
        self._check_table(feat, target, idx)
        nb = int(idx.shape[0]) if idx is not None else int(feat.shape[0])
        N.check(self._lib.pppm_corr_train_step(self._h, _stream(stream), _ptr(feat), _ptr(target), feat.shape[0],
                                               _ptr(idx), nb, ctypes.c_float(lr), _ptr(loss)),
                "pppm_corr_train_step")
        return loss


def wc_fold(f_sites: torch.Tensor, n_atoms: int, host_ptr=None, host_wc=None, jac_ptr=None, jac_wc=None,
            jac=None, out=None, status=None, stream=None) -> torch.Tensor:
    """Atom forces (n_atoms, 3) from site forces (atoms then WCs), Eq.
    DPLR:F_final: see pppm_wc_fold in include/pppm.h.  Index arrays: host_ptr
    int32 (n_atoms + 1), host_wc int32, jac_ptr int64 (n_atoms + 1), jac_wc
    int32, jac (nnz, 3, 3) in the dtype of f_sites; all CUDA tensors."""
    L = N.lib()
    f_sites = f_sites.contiguous()
    if f_sites.dtype not in (torch.float32, torch.float64) or not f_sites.is_cuda:
        raise ValueError("f_sites must be a float32 or float64 CUDA tensor")
    n_wc = f_sites.shape[0] - int(n_atoms)
    if n_wc < 0:
        raise ValueError("f_sites has fewer rows than n_atoms")
    for t, dt in ((host_ptr, torch.int32), (host_wc, torch.int32), (jac_ptr, torch.int64), (jac_wc, torch.int32),
                  (jac, f_sites.dtype)):
        if t is not None and (t.dtype != dt or not t.is_cuda or not t.is_contiguous()):
            raise ValueError(f"index/Jacobian arrays: expected contiguous CUDA {dt}")
    if out is None:
        out = torch.empty((int(n_atoms), 3), dtype=f_sites.dtype, device=f_sites.device)
    fn = L.pppm_wc_fold_f32 if f_sites.dtype == torch.float32 else L.pppm_wc_fold
    N.check(fn(_stream(stream), int(n_atoms), int(n_wc), _ptr(f_sites), _ptr(host_ptr), _ptr(host_wc),
               _ptr(jac_ptr), _ptr(jac_wc), _ptr(jac), _ptr(out), _ptr(status)), "pppm_wc_fold")
    return out
