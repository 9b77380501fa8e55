"""Python binding of the CUDA library: handle management and argument marshalling.

Every step of the computation runs in the library's CUDA kernels; this module only
passes pointers (PyTorch CUDA tensors provide device memory and the stream).
"""
from __future__ import annotations

import ctypes
import json
import os
import tempfile

import numpy as np
import torch

from . import _lib as L


class SoapGapError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"soapgap error {code}: {msg}")
        self.code = code


def _read_plan_cache(path: str) -> dict:
    """The plan cache's entries by problem class; empty when the file is missing, unreadable
    or not a JSON object."""
    try:
        with open(path) as f:
            known = json.load(f)
    except (OSError, ValueError):
        return {}
    return known if isinstance(known, dict) else {}


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    raise TypeError(type(t))


def _device_array(t, dtype, shape, name):
    """t itself if it is a contiguous CUDA tensor of this dtype and shape (the library reads
    it as a device array), else ValueError."""
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype
            and tuple(t.shape) == tuple(shape) and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor of shape {tuple(shape)}")
    return t


class Structures:
    """A batch of periodic structures: host metadata plus device positions/species."""

    def __init__(self, pos, cell, species, atom_offs, device="cuda"):
        self.atom_offs = np.ascontiguousarray(np.asarray(atom_offs, dtype=np.int64))
        self.cell = np.ascontiguousarray(np.asarray(cell, dtype=np.float64).reshape(-1, 3, 3))
        self.n_struct = int(self.cell.shape[0])
        if isinstance(pos, torch.Tensor):
            self.pos = pos.detach().to(device=device, dtype=torch.float64).contiguous()
        else:
            self.pos = torch.as_tensor(np.asarray(pos, dtype=np.float64), device=device).contiguous()
        if isinstance(species, torch.Tensor):
            self.species = species.to(device=device, dtype=torch.int32).contiguous()
        else:
            self.species = torch.as_tensor(np.asarray(species, dtype=np.int32), device=device).contiguous()
        self.n_atoms = int(self.pos.shape[0])
        if self.pos.dim() != 2 or self.pos.shape[1] != 3:
            raise ValueError("pos must be [n_atoms, 3]")
        if tuple(self.species.shape) != (self.n_atoms,):
            raise ValueError("species must be [n_atoms]")
        if self.atom_offs.shape != (self.n_struct + 1,):
            raise ValueError("atom_offs must be [n_struct + 1] for n_struct cells")

    @staticmethod
    def from_batch(b, device="cuda") -> "Structures":
        """From a synth.Batch (NumPy arrays)."""
        return Structures(b.pos, b.cell, b.species, b.atom_offs, device=device)

    def c_batch(self, pos=None, species=None) -> L.Batch:
        """The library's batch record.  Positions and species must still be contiguous CUDA
        tensors of their original shape and dtype: the library reads them as device arrays."""
        pos = self.pos if pos is None else pos
        species = self.species if species is None else species
        _device_array(pos, torch.float64, (self.n_atoms, 3), "pos")
        _device_array(species, torch.int32, (self.n_atoms,), "species")
        return L.Batch(self.n_struct, self.n_atoms, self.atom_offs.ctypes.data, self.cell.ctypes.data,
                       _ptr(pos), _ptr(species))


class SoapGap:
    """One descriptor/GAP configuration on the current CUDA device.

    precision: "mixed" (FP32 pair kernels, tensor-core GAP) or "fp64".
    """

    def __init__(self, *, r_cut, r_soft=None, sigma_r0=0.5, sigma_p0=None, alpha_r=0.0,
                 alpha_p=0.0, amp_a=1.0, n_f=4.0, central_weight=1.0, n_max=8, l_max=8,
                 n_species=1, precision="mixed", eq08_weight=False):
        self.lib = L.load()
        self.precision = precision
        self.dtype = torch.float32 if precision == "mixed" else torch.float64
        p = L.Params(r_cut, r_cut if r_soft is None else r_soft, sigma_r0,
                     sigma_r0 if sigma_p0 is None else sigma_p0, alpha_r, alpha_p, amp_a, n_f,
                     central_weight, n_max, l_max, n_species,
                     L.MIXED if precision == "mixed" else L.FP64, int(bool(eq08_weight)))
        self.params = p
        h = ctypes.c_void_p()
        rc = self.lib.soapgap_create(ctypes.byref(p), ctypes.byref(h))
        if rc != L.OK:
            raise SoapGapError(rc, "soapgap_create failed (see stderr)")
        self.h = h
        d = ctypes.c_int32()
        self._check(self.lib.soapgap_descriptor_dim(self.h, ctypes.byref(d)))
        self.dim = int(d.value)
        self.m = 0

    @classmethod
    def from_dict(cls, d: dict, precision="mixed"):
        keys = ("r_cut", "r_soft", "sigma_r0", "sigma_p0", "alpha_r", "alpha_p", "amp_a", "n_f",
                "central_weight", "n_max", "l_max", "n_species", "eq08_weight")
        return cls(precision=precision, **{k: d[k] for k in keys if k in d})

    def _check(self, rc):
        if rc != L.OK:
            msg = self.lib.soapgap_last_error(self.h)
            raise SoapGapError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self.lib.soapgap_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_model(self, q_sparse, alpha, zeta):
        qs = np.ascontiguousarray(np.asarray(q_sparse, dtype=np.float64))
        al = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64))
        if qs.ndim != 2 or qs.shape[1] != self.dim or al.shape != (qs.shape[0],):
            raise ValueError(f"q_sparse must be [M, {self.dim}] and alpha [M]")
        try:
            self._check(self.lib.soapgap_set_model(self.h, qs.ctypes.data, al.ctypes.data,
                                                   qs.shape[0], float(zeta)))
        except SoapGapError as e:
            if e.code != L.E_INVALID_ARG:
                self.m = 0          # the library dropped its previous model
            raise
        self.m = qs.shape[0]

    def compute(self, s: Structures, *, desc=False, energy=False, forces=False, virial=False,
                timing=False, asynchronous=False, stream=None):
        """Run one evaluation; returns a dict of CUDA tensors for the requested outputs.

        asynchronous=True: no allocation inside the library and no host synchronisation
        (capturable in a CUDA graph); needs an earlier synchronous call with the same batch
        shape, and device-side errors are reported by sync_status()."""
        dev = s.pos.device
        n, ns = s.n_atoms, s.n_struct
        flags = (L.DESC if desc else 0) | (L.ENERGY if energy else 0) | \
            (L.FORCES if forces else 0) | (L.VIRIAL if virial else 0) | \
            (L.TIMING if timing else 0) | (L.ASYNC if asynchronous else 0)
        out = {}
        if desc:
            out["q"] = torch.empty((n, self.dim), dtype=self.dtype, device=dev)
            out["pnorm"] = torch.empty((n,), dtype=self.dtype, device=dev)
        if energy:
            out["e_atom"] = torch.empty((n,), dtype=self.dtype, device=dev)
            out["e_struct"] = torch.empty((ns,), dtype=torch.float64, device=dev)
        if forces:
            out["forces"] = torch.empty((n, 3), dtype=torch.float64, device=dev)
        if virial:
            out["virial"] = torch.empty((ns, 3, 3), dtype=torch.float64, device=dev)
        st = (stream or torch.cuda.current_stream(dev)).cuda_stream
        b = s.c_batch()
        self._check(self.lib.soapgap_compute(
            self.h, ctypes.byref(b), flags, _ptr(out.get("q")), _ptr(out.get("pnorm")),
            _ptr(out.get("e_atom")), _ptr(out.get("e_struct")), _ptr(out.get("forces")),
            _ptr(out.get("virial")), st))
        return out

    def design(self, s: Structures, *, k_atom=False, k_struct=False, dk=False, timing=False,
               stream=None):
        """Rows of the sparse-GAP fitting matrices for the structures ``s`` against the
        sparse set of set_model (see soapgap_design): dict with k_atom [N, M],
        k_struct [S, M] and dk [N, 3, M] CUDA tensors as requested; a model with weights
        alpha has E = k_struct @ alpha and forces -dk @ alpha."""
        if self.m == 0:
            raise SoapGapError(L.E_STATE, "no sparse set: call set_model first")
        dev = s.pos.device
        n, ns, m = s.n_atoms, s.n_struct, self.m
        flags = (L.DESIGN_K if k_atom else 0) | (L.DESIGN_KSTRUCT if k_struct else 0) | \
            (L.DESIGN_DK if dk else 0) | (L.TIMING if timing else 0)
        out = {}
        if k_atom:
            out["k_atom"] = torch.empty((n, m), dtype=self.dtype, device=dev)
        if k_struct:
            out["k_struct"] = torch.empty((ns, m), dtype=torch.float64, device=dev)
        if dk:
            out["dk"] = torch.empty((n, 3, m), dtype=self.dtype, device=dev)
        st = (stream or torch.cuda.current_stream(dev)).cuda_stream
        b = s.c_batch()
        self._check(self.lib.soapgap_design(self.h, ctypes.byref(b), flags, _ptr(out.get("k_atom")),
                                            _ptr(out.get("k_struct")), _ptr(out.get("dk")), st))
        return out

    def design_times(self) -> dict:
        """Device milliseconds per stage of the last design(timing=True) call."""
        ms = np.zeros(L.N_DESIGN_STAGES)
        self._check(self.lib.soapgap_design_times(self.h, ms.ctypes.data))
        return dict(zip(L.DESIGN_STAGES, ms.tolist()))

    def kernel_rows(self, q: torch.Tensor, stream=None) -> torch.Tensor:
        """k[i, s] = (q_i . q_s)^zeta of descriptor rows q [n, D] (CUDA, the handle's dtype)
        against the sparse set; with the sparse rows themselves, the K_MM block."""
        if self.m == 0:
            raise SoapGapError(L.E_STATE, "no sparse set: call set_model first")
        q = q.to(self.dtype).contiguous()
        if q.ndim != 2 or q.shape[1] != self.dim:
            raise ValueError(f"q must be [n, {self.dim}]")
        _device_array(q, self.dtype, q.shape, "q")
        k = torch.empty((q.shape[0], self.m), dtype=self.dtype, device=q.device)
        st = (stream or torch.cuda.current_stream(q.device)).cuda_stream
        self._check(self.lib.soapgap_kernel_rows(self.h, _ptr(q), q.shape[0], _ptr(k), st))
        return k

    def set_gap_terms(self, terms: int):
        """FP16 products of the GAP energy on the tensor cores: 0 = chosen per model from
        the measured one-product error on the sparse rows (default), 1 or 3 = forced."""
        self._check(L.load().soapgap_set_gap_terms(self.h, int(terms)))

    def gap_terms(self) -> tuple[int, float]:
        """(products in use, measured one-product relative error of the sparse rows' energies)."""
        t = ctypes.c_int32(0)
        e = ctypes.c_double(0.0)
        self._check(L.load().soapgap_gap_terms(self.h, ctypes.byref(t), ctypes.byref(e)))
        return int(t.value), float(e.value)

    def set_skin(self, skin: float):
        """Verlet skin in A (0 disables neighbour-list reuse); see soapgap_set_skin."""
        self._check(self.lib.soapgap_set_skin(self.h, float(skin)))

    def last_rebuild(self) -> int:
        """1 if the last compute rebuilt the neighbour list, 0 if it reused it, -1 if the
        device decided (asynchronous call with a skin)."""
        r = ctypes.c_int32()
        self._check(self.lib.soapgap_last_rebuild(self.h, ctypes.byref(r)))
        return int(r.value)

    def verlet(self, s: "Structures", vel, forces, inv_mass, dt, drift: bool, stream=None):
        """Velocity-Verlet half step in place on s.pos and vel (see soapgap_verlet)."""
        n = s.n_atoms
        _device_array(vel, torch.float64, (n, 3), "vel")
        _device_array(forces, torch.float64, (n, 3), "forces")
        _device_array(inv_mass, torch.float64, (n,), "inv_mass")
        st = (stream or torch.cuda.current_stream(s.pos.device)).cuda_stream
        b = s.c_batch()
        self._check(self.lib.soapgap_verlet(self.h, ctypes.byref(b), _ptr(s.pos), _ptr(vel),
                                            _ptr(forces), _ptr(inv_mass), float(dt),
                                            1 if drift else 0, st))

    def sync_status(self, stream=None):
        """Wait for the stream; raise SoapGapError if the last asynchronous call flagged a
        device-side error (pair capacity, atom outside its cell, coincident atoms)."""
        st = (stream or torch.cuda.current_stream()).cuda_stream
        self._check(self.lib.soapgap_sync_status(self.h, st))

    PLAN_KEYS = ("adjoint_warps", "gap_forward", "gap_backward", "neighbour_sweep", "pair_forward")

    def _plan_cache_key(self, s: Structures) -> str:
        """Problem class of a batch as the library tunes it (after an evaluation of it), with
        the device and the model sizes that set the GAP products' shapes."""
        p = self.params
        n, nsp = s.n_atoms, p.n_species
        per_seg = self.pair_count() / max(1, n * nsp)
        batches = nsp * int(np.ceil(per_seg / 32.0))
        lg = int(np.ceil(np.log2(max(n, 1))))
        terms = self.gap_terms()[0] if self.precision == "mixed" else 0
        dev = torch.cuda.get_device_name(s.pos.device)
        return (f"{dev}|{self.precision}|n{p.n_max}l{p.l_max}sp{nsp}|M{self.m}|terms{terms}"
                f"|batches{batches}|lgN{lg}")

    def autotune(self, s: Structures, stream=None, cache: str | None = None) -> dict:
        """Pick the tile plan of this batch's problem class (soapgap_autotune): the adjoint
        variant, the tile configurations of the two GAP products, the neighbour sweep and the
        forward pair kernel.

        cache: path of a JSON file of earlier choices, keyed by device, precision, basis,
        species, model size, FP16 products and problem class.  A complete plan found there is
        installed without timing (soapgap_set_plan); an entry written by a version with fewer
        plan entries, or one the library rejects, is timed again and replaced.
        Returns {"adjoint_warps", "gap_forward", "gap_backward", "neighbour_sweep",
        "pair_forward", "cached"}."""
        st = (stream or torch.cuda.current_stream(s.pos.device)).cuda_stream
        b = s.c_batch()
        key = None
        if cache:
            self.compute(s, energy=True, forces=True, stream=stream)
            key = self._plan_cache_key(s)
            entry = _read_plan_cache(cache).get(key)
            vals = None
            if isinstance(entry, dict) and all(k in entry for k in self.PLAN_KEYS):
                try:
                    vals = [int(entry[k]) for k in self.PLAN_KEYS]
                except (TypeError, ValueError):
                    vals = None
            if vals is not None:
                arr = (ctypes.c_int32 * L.PLAN_LEN)(*vals)
                if self.lib.soapgap_set_plan(self.h, ctypes.byref(b), arr) == L.OK:
                    return dict(zip(self.PLAN_KEYS, vals), cached=True)
        arr = (ctypes.c_int32 * L.PLAN_LEN)()
        self._check(self.lib.soapgap_autotune(self.h, ctypes.byref(b), arr, st))
        plan = dict(zip(self.PLAN_KEYS, [int(x) for x in arr]))
        if cache:
            known = _read_plan_cache(cache)
            known[key] = plan
            d = os.path.dirname(os.path.abspath(cache))
            os.makedirs(d, exist_ok=True)
            fd, tmp = tempfile.mkstemp(dir=d, suffix=".json")
            with os.fdopen(fd, "w") as f:
                json.dump(known, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return dict(plan, cached=False)

    def set_plan(self, s: Structures, plan: dict):
        """Install a tile plan for this batch's problem class (soapgap_set_plan; the batch
        must have been evaluated on this handle)."""
        b = s.c_batch()
        arr = (ctypes.c_int32 * L.PLAN_LEN)(*[int(plan[k]) for k in self.PLAN_KEYS])
        self._check(self.lib.soapgap_set_plan(self.h, ctypes.byref(b), arr))

    def plan(self, s: Structures) -> dict:
        """The tile plan in use for this batch's problem class (soapgap_get_plan)."""
        b = s.c_batch()
        arr = (ctypes.c_int32 * L.PLAN_LEN)()
        self._check(self.lib.soapgap_get_plan(self.h, ctypes.byref(b), arr))
        return dict(zip(self.PLAN_KEYS, [int(x) for x in arr]))

    def backward(self, s: Structures, dE_dEstruct: torch.Tensor, virial=False, stream=None):
        """Gradient of sum_s w_s E_s with respect to positions (after an energy evaluation)."""
        dev = s.pos.device
        w = dE_dEstruct.to(device=dev, dtype=torch.float64).contiguous()
        if tuple(w.shape) != (s.n_struct,):
            raise ValueError(f"dE_dEstruct must be [n_struct] = [{s.n_struct}]")
        grad = torch.empty((s.n_atoms, 3), dtype=torch.float64, device=dev)
        vir = torch.empty((s.n_struct, 3, 3), dtype=torch.float64, device=dev) if virial else None
        st = (stream or torch.cuda.current_stream(dev)).cuda_stream
        b = s.c_batch()
        self._check(self.lib.soapgap_backward(self.h, ctypes.byref(b), _ptr(w), _ptr(grad),
                                              _ptr(vir), st))
        return (grad, vir) if virial else grad

    def compute_host(self, pos, cell, species, atom_offs, *, desc=False, energy=False,
                     forces=False, virial=False):
        """End-to-end call with host (NumPy) inputs and outputs."""
        pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64))
        species = np.ascontiguousarray(np.asarray(species, dtype=np.int32))
        atom_offs = np.ascontiguousarray(np.asarray(atom_offs, dtype=np.int64))
        cell = np.ascontiguousarray(np.asarray(cell, dtype=np.float64).reshape(-1, 3, 3))
        n, ns = pos.shape[0], cell.shape[0]
        npdt = np.float32 if self.precision == "mixed" else np.float64
        flags = (L.DESC if desc else 0) | (L.ENERGY if energy else 0) | \
            (L.FORCES if forces else 0) | (L.VIRIAL if virial else 0)
        out = {}
        if desc:
            out["q"] = np.empty((n, self.dim), npdt)
            out["pnorm"] = np.empty((n,), npdt)
        if energy:
            out["e_atom"] = np.empty((n,), npdt)
            out["e_struct"] = np.empty((ns,), np.float64)
        if forces:
            out["forces"] = np.empty((n, 3), np.float64)
        if virial:
            out["virial"] = np.empty((ns, 3, 3), np.float64)
        b = L.Batch(ns, n, atom_offs.ctypes.data, cell.ctypes.data, pos.ctypes.data,
                    species.ctypes.data)
        st = torch.cuda.current_stream().cuda_stream
        self._check(self.lib.soapgap_compute_host(
            self.h, ctypes.byref(b), flags, _ptr(out.get("q")), _ptr(out.get("pnorm")),
            _ptr(out.get("e_atom")), _ptr(out.get("e_struct")), _ptr(out.get("forces")),
            _ptr(out.get("virial")), st))
        return out

    def stage_times(self) -> dict:
        """Device milliseconds per stage of the last compute(timing=True) call."""
        ms = np.zeros(L.N_STAGES)
        self._check(self.lib.soapgap_stage_times(self.h, ms.ctypes.data))
        return dict(zip(L.STAGES, ms.tolist()))

    def launch_count(self) -> int:
        """Kernels launched by the last compute/backward call."""
        n = ctypes.c_int64()
        self._check(self.lib.soapgap_last_launch_count(self.h, ctypes.byref(n)))
        return int(n.value)

    def pair_count(self) -> int:
        n = ctypes.c_int64()
        self._check(self.lib.soapgap_last_pair_count(self.h, ctypes.byref(n)))
        return int(n.value)

    def pairs(self):
        """Pair list of the last compute call: (centre, neighbour, shift[P, 3]) as NumPy."""
        p = self.pair_count()
        i = np.empty(max(p, 1), np.int32)
        j = np.empty(max(p, 1), np.int32)
        s = np.empty((max(p, 1), 3), np.int32)
        self._check(self.lib.soapgap_export_pairs(self.h, p, i.ctypes.data, j.ctypes.data,
                                                  s.ctypes.data))
        return i[:p], j[:p], s[:p]


def measure_alu_peak(kind: str = "fp32", stream=None) -> tuple[float, int]:
    """Measured FMA throughput of the current device in TFLOP/s and its SM count
    (soapgap_measure_alu_peak; kind "fp32" or "fp64")."""
    lib = L.load()
    k = {"fp32": L.PEAK_FP32_FMA, "fp64": L.PEAK_FP64_FMA}[kind]
    tf = ctypes.c_double(0.0)
    sms = ctypes.c_int32(0)
    st = (stream or torch.cuda.current_stream()).cuda_stream
    rc = lib.soapgap_measure_alu_peak(k, ctypes.byref(tf), ctypes.byref(sms), st)
    if rc != L.OK:
        raise SoapGapError(rc, f"soapgap_measure_alu_peak({kind}) failed")
    return float(tf.value), int(sms.value)


class SoapGapEnergy(torch.autograd.Function):
    """E_struct = GAP energies of a batch, differentiable with respect to positions.

    forward(pos [N,3] CUDA float64, model: SoapGap, s: Structures) -> E_struct [S] float64.
    The backward pass is the library's adjoint kernel chain (soapgap_backward).
    """

    @staticmethod
    def forward(ctx, pos, model: SoapGap, s: Structures):
        s2 = Structures(pos.detach(), s.cell, s.species, s.atom_offs, device=pos.device)
        out = model.compute(s2, energy=True)
        ctx.model = model
        ctx.s = s2
        return out["e_struct"]

    @staticmethod
    def backward(ctx, grad_e):
        grad = ctx.model.backward(ctx.s, grad_e.detach())
        return grad, None, None


class CapturedEvaluation:
    """One evaluation of a fixed batch shape captured in a CUDA graph.

    The constructor makes one synchronous call (sizing the workspace), then captures an
    asynchronous call; replay() re-runs the whole evaluation (neighbour list included) on
    the current contents of s.pos / s.species and returns the same output tensors, updated
    in place.  Call model.sync_status() after replays to surface device-side errors.
    Capture again after model.set_model: the graph holds the buffers of the model it saw."""

    def __init__(self, model: SoapGap, s: Structures, **outputs):
        self.model, self.s = model, s
        model.compute(s, **outputs)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.out = model.compute(s, asynchronous=True, **outputs)

    def replay(self):
        self.graph.replay()
        return self.out


AMU_A2_PER_FS2_IN_EV = 103.642697  # 1 amu A^2 / fs^2 in eV


class VelocityVerlet:
    """Microcanonical molecular dynamics around the evaluation (units A, fs, amu, eV).

    Each step: kick + drift (library kernel), forces and energies at the new positions
    (soapgap_compute; the neighbour list is reused while the model's Verlet skin allows),
    closing kick.  With capture=True one step is captured in a CUDA graph and replayed.
    """

    def __init__(self, model: SoapGap, s: Structures, masses, dt: float, vel=None,
                 capture: bool = False):
        self.model, self.s, self.dt = model, s, float(dt)
        dev = s.pos.device
        m = torch.as_tensor(np.asarray(masses, dtype=np.float64), device=dev).reshape(-1)
        if m.numel() == 1:
            m = m.expand(s.n_atoms).contiguous()
        self.mass = m
        self.inv_mass = (1.0 / m).contiguous()
        self.vel = (torch.zeros((s.n_atoms, 3), dtype=torch.float64, device=dev) if vel is None
                    else torch.as_tensor(vel, dtype=torch.float64, device=dev).clone().contiguous())
        self.out = model.compute(s, energy=True, forces=True)
        self.f = self.out["forces"].clone()     # forces of the current positions
        self.graph = None
        if capture:
            # the synchronous compute above sized the workspace of the captured calls
            torch.cuda.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph):
                self._step(asynchronous=True)

    def _step(self, asynchronous):
        self.model.verlet(self.s, self.vel, self.f, self.inv_mass, self.dt, drift=True)
        self.out = self.model.compute(self.s, energy=True, forces=True, asynchronous=asynchronous)
        self.f.copy_(self.out["forces"])
        self.model.verlet(self.s, self.vel, self.f, self.inv_mass, self.dt, drift=False)

    def step(self, n: int = 1):
        for _ in range(n):
            if self.graph is not None:
                self.graph.replay()
            else:
                self._step(asynchronous=False)
        return self

    def potential_energy(self) -> float:
        return float(self.out["e_struct"].sum())

    def kinetic_energy(self) -> float:
        return float(0.5 * AMU_A2_PER_FS2_IN_EV * (self.mass[:, None] * self.vel ** 2).sum())
