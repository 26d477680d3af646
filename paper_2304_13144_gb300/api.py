"""Python binding of the C ABI in include/mtp.h (argument marshalling only).

Every function mirrors the C entry point of the same name; torch tensors supply device
memory and the current CUDA stream.  The CUDA library must have been built
(paper_2304_13144_gb300.build.build()); importing this module without it raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmtp.so")

MTP_FP64 = 0
MTP_MIXED = 1
MTP_GRADE_NEIGHBORHOOD = 0
MTP_GRADE_CONFIGURATION = 1
STATUS = {0: "MTP_OK", 1: "MTP_ERR_ARG", 2: "MTP_ERR_CUDA", 3: "MTP_ERR_CAPACITY", 4: "MTP_ERR_SINGULAR",
          5: "MTP_ERR_GEOMETRY", 6: "MTP_ERR_NUMERIC", 7: "MTP_ERR_UNSUPPORTED", 8: "MTP_ERR_TIMEOUT"}


class MtpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class mtp_desc(ctypes.Structure):
    _fields_ = [("n_types", ctypes.c_int32), ("lev_max", ctypes.c_int32), ("n_q", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("r_min", ctypes.c_double), ("r_cut", ctypes.c_double)]


class mtp_sizes(ctypes.Structure):
    _fields_ = [("n_params", ctypes.c_int64), ("n_lin", ctypes.c_int32), ("n_rad", ctypes.c_int32),
                ("n_moments", ctypes.c_int32), ("n_mom_comps", ctypes.c_int32), ("n_values", ctypes.c_int32),
                ("n_triples", ctypes.c_int32), ("nu_max", ctypes.c_int32), ("n_gauge", ctypes.c_int32)]


class mtp_batch(ctypes.Structure):
    _fields_ = [("n_cfg", ctypes.c_int32), ("reserved", ctypes.c_int32), ("atom_offset", ctypes.c_void_p),
                ("pos", ctypes.c_void_p), ("type", ctypes.c_void_p), ("cell", ctypes.c_void_p),
                ("pbc", ctypes.c_void_p)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_SIGS = {
    "mtp_version": (ctypes.c_char_p, []),
    "mtp_last_error": (ctypes.c_char_p, []),
    "mtp_describe": (ctypes.c_int, [_P, _P]),
    "mtp_describe_basis": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "mtp_describe_schedule": (ctypes.c_int, [_P] * 8),
    "mtp_gauge_directions": (ctypes.c_int, [_P, _P, _I64, _P]),
    "mtp_load": (ctypes.c_int, [_P, _P, _I64, _P]),
    "mtp_free_model": (None, [_P]),
    "mtp_num_params": (_I64, [_P]),
    "mtp_model_sizes": (ctypes.c_int, [_P, _P]),
    "mtp_set_params": (ctypes.c_int, [_P, _P, _I64]),
    "mtp_set_active_set": (ctypes.c_int, [_P, _P, _I64, _P]),
    "mtp_get_active_inverse": (ctypes.c_int, [_P, _P, _P]),
    "mtp_get_active_set": (ctypes.c_int, [_P, _P, _P]),
    "mtp_save": (ctypes.c_int, [_P, _P, _I64, _P, _P]),
    "mtp_restore": (ctypes.c_int, [_P, _I64, _P, _P]),
    "mtp_debug_inject": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
    "mtp_sync": (ctypes.c_int, [_P, _P]),
    "mtp_set_mixed_pass": (ctypes.c_int, [_P, ctypes.c_int]),
    "mtp_get_mixed_pass": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "mtp_set_split_shape": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "mtp_get_split_shape": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "mtp_measure_peak": (ctypes.c_int, [ctypes.c_int, _P, _P, _P]),
    "mtp_autotune": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P, _P]),
    "mtp_fit_bfgs": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P, _P, _D, _D, _D, _I64, _D, _P, _P, _P]),
    "mtp_fit_errors": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P, _P, _P, _P]),
    "mtp_get_params": (ctypes.c_int, [_P, _P, _I64]),
    "mtp_cut_clusters": (ctypes.c_int, [_P, _P, _I64, _D, _P, _P, _P, _P, _I64, _P, _P]),
    "mtp_config_rows": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P]),
    "mtp_energy_vjp": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P, _P, _P, _P]),
    "mtp_config_grade": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, _D, _D, _P, _P, _P, _P]),
    "mtp_maxvol": (ctypes.c_int, [_P, _P, _I64, _D, _I64, _P, _P, _P]),
    "mtp_build_neighbors": (ctypes.c_int, [_P, _P, _P, _P]),
    "mtp_free_nbr": (None, [_P]),
    "mtp_nbr_size": (ctypes.c_int, [_P, _P, _P]),
    "mtp_nbr_export": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "mtp_nbr_reverse": (ctypes.c_int, [_P, _P, _P]),
    "mtp_energy_forces_stress": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P, _P, _P, _P]),
    "mtp_energy_forces_stress_atoms": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P, _P, _P, _P, _P]),
    "mtp_energy_forces_stress_noalloc": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P, _P, _P, _P]),
    "mtp_param_rows": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _I64, _P, _P]),
    "mtp_grade": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _D, _P, _P, _P, _P, _P]),
    "mtp_step": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P, _P, _P, _D, _P, _P, _P, _P, _P]),
    "mtp_extract_neighborhoods": (ctypes.c_int, [_P, _P, _P, _I64, _P, _P, _P, _P, _I64, _P, _P]),
    "mtp_train_step": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P, _P, _D, _D, _D, _P, _P, _P]),
    "mtp_profiler_enable": (ctypes.c_int, [ctypes.c_int]),
    "mtp_profiler_read": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libmtp.so (raises if it was not built: there is no CPU fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} missing (run paper_2304_13144_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st):
    if st != 0:
        raise MtpError(st, lib().mtp_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    raise TypeError(type(t))


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def make_desc(n_types, lev_max, n_q=8, r_min=2.0, r_cut=5.0):
    return mtp_desc(int(n_types), int(lev_max), int(n_q), 0, float(r_min), float(r_cut))


# ------------------------------------------------------------------------------------
# host-only descriptions
# ------------------------------------------------------------------------------------

def mtp_describe(desc) -> dict:
    out = mtp_sizes()
    _check(lib().mtp_describe(ctypes.byref(desc), ctypes.byref(out)))
    return {k: getattr(out, k) for k, _ in mtp_sizes._fields_}


def mtp_describe_basis(desc):
    n = mtp_describe(desc)["n_lin"]
    P = np.zeros(n, np.int32)
    mu = np.zeros((n, 4), np.int32)
    nu = np.zeros((n, 4), np.int32)
    ed = np.zeros((n, 6), np.int32)
    _check(lib().mtp_describe_basis(ctypes.byref(desc), _ptr(P), _ptr(mu), _ptr(nu), _ptr(ed)))
    full = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    basis = []
    for a in range(n):
        p = int(P[a])
        labels = tuple((int(mu[a, k]), int(nu[a, k])) for k in range(p))
        edges = tuple(int(ed[a, full.index((i, j))]) for i in range(p) for j in range(i + 1, p))
        basis.append((labels, edges))
    return basis


def mtp_describe_schedule(desc) -> dict:
    sz = mtp_describe(desc)
    nm, nv, nt, nl = sz["n_mom_comps"], sz["n_values"], sz["n_triples"], sz["n_lin"]
    out = {"comp_mu": np.zeros(nm, np.int32), "comp_exp": np.zeros((nm, 3), np.int32),
           "dst_ptr": np.zeros(nv - nm + 1, np.int32), "tri_a": np.zeros(max(nt, 1), np.int32),
           "tri_b": np.zeros(max(nt, 1), np.int32), "tri_c": np.zeros(max(nt, 1), np.float64),
           "basis_idx": np.zeros(nl, np.int32)}
    _check(lib().mtp_describe_schedule(ctypes.byref(desc), *[_ptr(out[k]) for k in
                                                             ("comp_mu", "comp_exp", "dst_ptr", "tri_a", "tri_b",
                                                              "tri_c", "basis_idx")]))
    out["sizes"] = sz
    return out


def mtp_gauge_directions(desc, theta):
    theta = np.ascontiguousarray(theta, np.float64)
    sz = mtp_describe(desc)
    D = np.zeros((sz["n_gauge"], sz["n_params"]))
    _check(lib().mtp_gauge_directions(ctypes.byref(desc), _ptr(theta), theta.size, _ptr(D)))
    return D


# ------------------------------------------------------------------------------------
# handles
# ------------------------------------------------------------------------------------

class Model:
    """Owns an mtp_model*."""

    def __init__(self, desc, theta):
        self.desc = desc
        theta = np.ascontiguousarray(theta, np.float64)
        h = ctypes.c_void_p()
        _check(lib().mtp_load(ctypes.byref(desc), _ptr(theta), theta.size, ctypes.byref(h)))
        self.h = h
        self.sizes = self.model_sizes()

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.mtp_free_model(self.h)
            self.h = None

    @property
    def n_params(self):
        return int(lib().mtp_num_params(self.h))

    def model_sizes(self):
        out = mtp_sizes()
        _check(lib().mtp_model_sizes(self.h, ctypes.byref(out)))
        return {k: getattr(out, k) for k, _ in mtp_sizes._fields_}


class Batch:
    """Device copies of a batch (see synth.py for the dict layout) and the mtp_batch struct."""

    def __init__(self, b, device="cuda"):
        self.atom_offset = torch.as_tensor(np.ascontiguousarray(b["atom_offset"], np.int64), device=device)
        self.pos = torch.as_tensor(np.ascontiguousarray(b["pos"], np.float64), device=device)
        self.type = torch.as_tensor(np.ascontiguousarray(b["type"], np.int32), device=device)
        self.cell = torch.as_tensor(np.ascontiguousarray(b["cell"], np.float64).reshape(-1, 9), device=device)
        self.pbc = torch.as_tensor(np.ascontiguousarray(b["pbc"], np.uint8).reshape(-1, 3), device=device)
        self.n_cfg = int(self.atom_offset.numel() - 1)
        self.n_atoms = int(b["atom_offset"][-1])
        self.refresh()

    def refresh(self):
        self.c = mtp_batch(self.n_cfg, 0, self.atom_offset.data_ptr(), self.pos.data_ptr(), self.type.data_ptr(),
                           self.cell.data_ptr(), self.pbc.data_ptr())
        return self


class Neighbors:
    """Owns an mtp_nbr*."""

    def __init__(self):
        self.h = ctypes.c_void_p()

    def __del__(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.mtp_free_nbr(self.h)
            self.h = ctypes.c_void_p()

    def size(self):
        na, npairs = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().mtp_nbr_size(self.h, ctypes.byref(na), ctypes.byref(npairs)))
        return na.value, npairs.value


# ------------------------------------------------------------------------------------
# entry points
# ------------------------------------------------------------------------------------

def mtp_load(desc, theta) -> Model:
    return Model(desc, theta)


def mtp_set_params(model: Model, theta):
    theta = np.ascontiguousarray(theta, np.float64)
    _check(lib().mtp_set_params(model.h, _ptr(theta), theta.size))


def mtp_set_active_set(model: Model, A: torch.Tensor, stream=None):
    A = A.to(dtype=torch.float64).contiguous()
    _check(lib().mtp_set_active_set(model.h, _ptr(A), A.shape[0], _stream(stream)))


def mtp_get_active_inverse(model: Model, stream=None):
    m = model.n_params
    out = torch.empty((m, m), dtype=torch.float64, device="cuda")
    _check(lib().mtp_get_active_inverse(model.h, _ptr(out), _stream(stream)))
    return out


def mtp_get_active_set(model: Model, stream=None):
    m = model.n_params
    out = torch.empty((m, m), dtype=torch.float64, device="cuda")
    _check(lib().mtp_get_active_set(model.h, _ptr(out), _stream(stream)))
    return out


def mtp_maxvol(model: Model, B: torch.Tensor, eps=1e-3, max_swaps=1_000_000, stream=None):
    """MaxVol update of the model's active set with candidate rows B (n x m): returns
    (source[m] int64 device tensor, number of swaps)."""
    B = B.to(device="cuda", dtype=torch.float64).contiguous()
    n = int(B.shape[0]) if B.dim() == 2 else 0
    source = torch.empty(model.n_params, dtype=torch.int64, device="cuda")
    swaps = ctypes.c_int64()
    _check(lib().mtp_maxvol(model.h, _ptr(B) if n else None, n, float(eps), int(max_swaps), _ptr(source),
                            ctypes.byref(swaps), _stream(stream)))
    return source, swaps.value


def mtp_build_neighbors(model: Model, batch: Batch, nbr: Neighbors | None = None, stream=None) -> Neighbors:
    nbr = nbr or Neighbors()
    _check(lib().mtp_build_neighbors(model.h, ctypes.byref(batch.c), ctypes.byref(nbr.h), _stream(stream)))
    return nbr


def mtp_nbr_export(nbr: Neighbors, batch: Batch, want_r=True, stream=None):
    na, npairs = nbr.size()
    off = torch.empty(na + 1, dtype=torch.int64, device="cuda")
    j = torch.empty(max(npairs, 1), dtype=torch.int32, device="cuda")
    img = torch.empty((max(npairs, 1), 3), dtype=torch.int32, device="cuda")
    r = torch.empty((max(npairs, 1), 3), dtype=torch.float64, device="cuda") if want_r else None
    _check(lib().mtp_nbr_export(nbr.h, ctypes.byref(batch.c), _ptr(off), _ptr(j), _ptr(img),
                                _ptr(r) if want_r else None, _stream(stream)))
    out = {"off": off, "j": j[:npairs], "img": img[:npairs]}
    if want_r:
        out["r"] = r[:npairs]
    return out


def mtp_nbr_reverse(nbr: Neighbors, stream=None):
    """rev[p]: position of the reverse pair (j -> i, -n) of pair p = (i -> j, n)."""
    _, npairs = nbr.size()
    rev = torch.empty(max(npairs, 1), dtype=torch.int32, device="cuda")
    _check(lib().mtp_nbr_reverse(nbr.h, _ptr(rev), _stream(stream)))
    return rev[:npairs]


def _prec(p):
    if p in ("fp64", MTP_FP64):
        return MTP_FP64
    if p in ("mixed", MTP_MIXED):
        return MTP_MIXED
    raise ValueError(p)


def mtp_energy_forces_stress(model, batch, nbr, prec="mixed", energy=None, site_energy=None, forces=None,
                             virial=None, want=("energy", "forces", "virial", "site_energy"), stream=None):
    dev = "cuda"
    N, K = batch.n_atoms, batch.n_cfg
    if energy is None and "energy" in want:
        energy = torch.empty(K, dtype=torch.float64, device=dev)
    if site_energy is None and "site_energy" in want:
        site_energy = torch.empty(N, dtype=torch.float64, device=dev)
    if forces is None and "forces" in want:
        forces = torch.empty((N, 3), dtype=torch.float64, device=dev)
    if virial is None and "virial" in want:
        virial = torch.empty((K, 3, 3), dtype=torch.float64, device=dev)
    _check(lib().mtp_energy_forces_stress(model.h, ctypes.byref(batch.c), nbr.h, _prec(prec), _ptr(energy),
                                          _ptr(site_energy), _ptr(forces), _ptr(virial), _stream(stream)))
    return {"energy": energy, "site_energy": site_energy, "forces": forces, "virial": virial}


def mtp_energy_forces_stress_atoms(model, batch, nbr, prec="mixed", stream=None):
    """Energies, site energies, forces, virial and per-atom virials W_i (N, 3, 3)."""
    N, K = batch.n_atoms, batch.n_cfg
    out = {"energy": torch.empty(K, dtype=torch.float64, device="cuda"),
           "site_energy": torch.empty(N, dtype=torch.float64, device="cuda"),
           "forces": torch.empty((N, 3), dtype=torch.float64, device="cuda"),
           "virial": torch.empty((K, 3, 3), dtype=torch.float64, device="cuda"),
           "site_virial": torch.empty((N, 3, 3), dtype=torch.float64, device="cuda")}
    _check(lib().mtp_energy_forces_stress_atoms(model.h, ctypes.byref(batch.c), nbr.h, _prec(prec),
                                                *[_ptr(out[k]) for k in ("energy", "site_energy", "forces", "virial",
                                                                        "site_virial")], _stream(stream)))
    return out


def mtp_energy_forces_stress_noalloc(model, batch, nbr, prec="mixed",
                                     want=("energy", "forces", "virial", "site_energy"), stream=None):
    """Allocation-free energies/forces/virial: the library allocates nothing (the requested
    outputs are allocated here by torch, before the call; the others are passed as NULL)."""
    N, K = batch.n_atoms, batch.n_cfg
    energy = torch.empty(K, dtype=torch.float64, device="cuda") if "energy" in want else None
    site_energy = torch.empty(N, dtype=torch.float64, device="cuda") if "site_energy" in want else None
    forces = torch.empty((N, 3), dtype=torch.float64, device="cuda") if "forces" in want else None
    virial = torch.empty((K, 3, 3), dtype=torch.float64, device="cuda") if "virial" in want else None
    _check(lib().mtp_energy_forces_stress_noalloc(model.h, ctypes.byref(batch.c), nbr.h, _prec(prec), _ptr(energy),
                                                  _ptr(site_energy), _ptr(forces), _ptr(virial), _stream(stream)))
    return {"energy": energy, "site_energy": site_energy, "forces": forces, "virial": virial}


def mtp_param_rows(model, batch, nbr, prec="fp64", atoms=None, stream=None):
    n = batch.n_atoms if atoms is None else int(atoms.numel())
    rows = torch.empty((n, model.n_params), dtype=torch.float64, device="cuda")
    if atoms is not None:
        atoms = atoms.to(device="cuda", dtype=torch.int64).contiguous()
    _check(lib().mtp_param_rows(model.h, ctypes.byref(batch.c), nbr.h, _prec(prec), _ptr(atoms), n, _ptr(rows),
                                _stream(stream)))
    return rows


def mtp_grade(model, batch, nbr, prec="mixed", threshold=2.0, stream=None):
    N = batch.n_atoms
    gamma = torch.empty(N, dtype=torch.float64, device="cuda")
    argmax = torch.empty(N, dtype=torch.int32, device="cuda")
    flagged = torch.empty(max(N, 1), dtype=torch.int32, device="cuda")
    n_flagged = torch.zeros(1, dtype=torch.int64, device="cuda")
    _check(lib().mtp_grade(model.h, ctypes.byref(batch.c), nbr.h, _prec(prec), float(threshold), _ptr(gamma),
                           _ptr(argmax), _ptr(flagged), _ptr(n_flagged), _stream(stream)))
    return {"gamma": gamma, "argmax": argmax, "flagged": flagged, "n_flagged": n_flagged}


def mtp_step(model, batch, nbr, prec="mixed", threshold=2.0, out=None, grade=True, stream=None):
    N, K = batch.n_atoms, batch.n_cfg
    if out is None:
        out = {"energy": torch.empty(K, dtype=torch.float64, device="cuda"),
               "site_energy": None,
               "forces": torch.empty((N, 3), dtype=torch.float64, device="cuda"),
               "virial": torch.empty((K, 3, 3), dtype=torch.float64, device="cuda")}
        if grade:
            out.update({"gamma": torch.empty(N, dtype=torch.float64, device="cuda"),
                        "argmax": torch.empty(N, dtype=torch.int32, device="cuda"),
                        "flagged": torch.empty(max(N, 1), dtype=torch.int32, device="cuda"),
                        "n_flagged": torch.zeros(1, dtype=torch.int64, device="cuda")})
    g = out.get("gamma")
    _check(lib().mtp_step(model.h, ctypes.byref(batch.c), nbr.h, _prec(prec), _ptr(out.get("energy")),
                          _ptr(out.get("site_energy")), _ptr(out.get("forces")), _ptr(out.get("virial")),
                          float(threshold), _ptr(g), _ptr(out.get("argmax")), _ptr(out.get("flagged")),
                          _ptr(out.get("n_flagged")), _stream(stream)))
    return out


def mtp_config_rows(model, batch, nbr, prec="fp64", stream=None):
    rows = torch.empty((batch.n_cfg, model.n_params), dtype=torch.float64, device="cuda")
    _check(lib().mtp_config_rows(model.h, ctypes.byref(batch.c), nbr.h, _prec(prec), _ptr(rows), _stream(stream)))
    return rows


def mtp_energy_vjp(model, batch, nbr, gE, forces=None, want_pos=True, want_theta=True, prec="fp64", stream=None):
    """(g_pos, g_theta): the vector-Jacobian product of the configuration energies for the
    cotangent gE (n_cfg,); either output is None when not requested."""
    gE = gE.to(device="cuda", dtype=torch.float64).contiguous()
    g_pos = torch.empty((batch.n_atoms, 3), dtype=torch.float64, device="cuda") if want_pos else None
    g_theta = torch.empty(model.n_params, dtype=torch.float64, device="cuda") if want_theta else None
    F = forces.contiguous() if forces is not None else None
    _check(lib().mtp_energy_vjp(model.h, ctypes.byref(batch.c), nbr.h, _prec(prec), _ptr(gE), _ptr(F), _ptr(g_pos),
                                _ptr(g_theta), _stream(stream)))
    return g_pos, g_theta


def mtp_config_grade(model, batch, nbr, prec="fp64", mode="neighborhood", gamma_save=2.0, gamma_break=10.0,
                     stream=None):
    """Per-configuration grade, the worst atom (neighborhood mode) or active row (configuration
    mode), and the class 0 continue / 1 save / 2 stop."""
    md = {"neighborhood": MTP_GRADE_NEIGHBORHOOD, "configuration": MTP_GRADE_CONFIGURATION}[mode]
    K = batch.n_cfg
    gamma = torch.empty(K, dtype=torch.float64, device="cuda")
    worst = torch.empty(K, dtype=torch.int64, device="cuda")
    cls = torch.empty(K, dtype=torch.int32, device="cuda")
    _check(lib().mtp_config_grade(model.h, ctypes.byref(batch.c), nbr.h, _prec(prec), md, float(gamma_save),
                                  float(gamma_break), _ptr(gamma), _ptr(worst), _ptr(cls), _stream(stream)))
    return {"gamma": gamma, "worst": worst, "class": cls}


def mtp_extract_neighborhoods(nbr, batch, idx: torch.Tensor, capacity=None, stream=None):
    idx = idx.to(device="cuda", dtype=torch.int32).contiguous()
    n = int(idx.numel())
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    total = ctypes.c_int64()
    if capacity is None:
        # ask for the size first
        st = lib().mtp_extract_neighborhoods(nbr.h, ctypes.byref(batch.c), _ptr(idx), n, _ptr(off), None, None,
                                             None, 0, ctypes.byref(total), _stream(stream))
        if st not in (0, 3):
            _check(st)
        capacity = total.value
    r = torch.empty((max(capacity, 1), 3), dtype=torch.float64, device="cuda")
    ty = torch.empty(max(capacity, 1), dtype=torch.int32, device="cuda")
    j = torch.empty(max(capacity, 1), dtype=torch.int32, device="cuda")
    _check(lib().mtp_extract_neighborhoods(nbr.h, ctypes.byref(batch.c), _ptr(idx), n, _ptr(off), _ptr(r),
                                           _ptr(ty), _ptr(j), capacity, ctypes.byref(total), _stream(stream)))
    t = total.value
    return {"off": off, "r": r[:t], "type": ty[:t], "j": j[:t]}


def mtp_cut_clusters(batch, centers: torch.Tensor, radius=8.0, stream=None):
    """Non-periodic clusters of radius `radius` around the center atoms: CSR offsets and, per
    cluster atom, position relative to its center, species and source atom."""
    centers = centers.to(device="cuda", dtype=torch.int64).contiguous()
    n = int(centers.numel())
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    total = ctypes.c_int64()
    _check(lib().mtp_cut_clusters(ctypes.byref(batch.c), _ptr(centers) if n else None, n, float(radius), _ptr(off),
                                  None, None, None, 0, ctypes.byref(total), _stream(stream)))
    t = total.value
    pos = torch.empty((max(t, 1), 3), dtype=torch.float64, device="cuda")
    ty = torch.empty(max(t, 1), dtype=torch.int32, device="cuda")
    src = torch.empty(max(t, 1), dtype=torch.int64, device="cuda")
    _check(lib().mtp_cut_clusters(ctypes.byref(batch.c), _ptr(centers) if n else None, n, float(radius), _ptr(off),
                                  _ptr(pos), _ptr(ty), _ptr(src), t, ctypes.byref(total), _stream(stream)))
    return {"off": off, "pos": pos[:t], "type": ty[:t], "src": src[:t]}


def mtp_train_step(model, batch, nbr, E_ref, F_ref, W_ref=None, w_e=1.0, w_f=0.01, w_s=0.0, prec="fp64",
                   stream=None):
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    grad = torch.empty(model.n_params, dtype=torch.float64, device="cuda")
    E_ref = E_ref.to(device="cuda", dtype=torch.float64).contiguous()
    F_ref = F_ref.to(device="cuda", dtype=torch.float64).contiguous()
    if W_ref is not None:
        W_ref = W_ref.to(device="cuda", dtype=torch.float64).contiguous()
    _check(lib().mtp_train_step(model.h, ctypes.byref(batch.c), nbr.h, _prec(prec), _ptr(E_ref), _ptr(F_ref),
                                _ptr(W_ref), float(w_e), float(w_f), float(w_s), _ptr(loss), _ptr(grad),
                                _stream(stream)))
    return loss, grad


def mtp_autotune(model, batch, nbr, prec="mixed", stream=None):
    """Pick the per-neighborhood kernel's warps per block by timing; returns (warps, ms)."""
    w, ms = ctypes.c_int32(), ctypes.c_double()
    _check(lib().mtp_autotune(model.h, ctypes.byref(batch.c), nbr.h, _prec(prec), ctypes.byref(w), ctypes.byref(ms),
                              _stream(stream)))
    return w.value, ms.value


def mtp_set_mixed_pass(model, p):
    """0 automatic, 1 single kernel, 2 three kernels (or the names "auto", "single", "split")."""
    p = {"auto": 0, "single": 1, "split": 2}.get(p, p)
    _check(lib().mtp_set_mixed_pass(model.h, int(p)))


def mtp_set_split_shape(model, warps_pair=0, nb_contract=0, unroll=0, schedule=0):
    """schedule: 0 automatic, 1 shared memory, 2 streamed through a shared ring, 3 tensor memory."""
    _check(lib().mtp_set_split_shape(model.h, int(warps_pair), int(nb_contract), int(unroll), int(schedule)))


def mtp_get_split_shape(model):
    """(warps_pair, nb_contract, unroll, schedule setting, placement the last pass used: 1, 2 or 3)."""
    v = [ctypes.c_int32() for _ in range(5)]
    _check(lib().mtp_get_split_shape(model.h, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def mtp_get_mixed_pass(model):
    """(setting, pass in use: 1 or 2, split warps, split neighborhoods per warp)."""
    v = [ctypes.c_int32() for _ in range(4)]
    _check(lib().mtp_get_mixed_pass(model.h, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def mtp_get_launch_shape(model):
    """The autotuner's shapes kept in the model: (warps_fast, fwd_global, warps_generic)."""
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().mtp_get_launch_shape(model.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def mtp_save(model, stream=None) -> bytes:
    """Checkpoint of the model (descriptor, theta, active set) as bytes."""
    size = ctypes.c_int64()
    _check(lib().mtp_save(model.h, None, 0, ctypes.byref(size), _stream(stream)))
    buf = ctypes.create_string_buffer(size.value)
    _check(lib().mtp_save(model.h, buf, size.value, ctypes.byref(size), _stream(stream)))
    return buf.raw[:size.value]


def mtp_restore(blob: bytes, stream=None) -> Model:
    """A new model from a checkpoint made by mtp_save."""
    m = Model.__new__(Model)
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    _check(lib().mtp_restore(buf, len(blob), ctypes.byref(h), _stream(stream)))
    m.h = h
    m.desc = None
    m.sizes = m.model_sizes()
    return m


MTP_FAULT_DEVICE_ALLOC = 1
MTP_FAULT_NEIGHBOR_OVERFLOW = 2
MTP_FAULT_GRADE_WAIT = 3


def mtp_debug_inject(fault, count):
    """Arm a host-side fault for the next `count` events (0 disarms)."""
    _check(lib().mtp_debug_inject(int(fault), int(count)))


def mtp_sync(model, stream=None):
    """Synchronise the stream; raise the device-side error latched by earlier asynchronous calls."""
    _check(lib().mtp_sync(model.h, _stream(stream)))


def mtp_measure_peak(kind, stream=None):
    """(TFLOP/s, ms) of the library's microbenchmark: kind "fp32_fma", "fp64_fma" or "tf32_mma"."""
    k = {"fp32_fma": 0, "fp64_fma": 1, "tf32_mma": 2}[kind]
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().mtp_measure_peak(k, ctypes.byref(tf), ctypes.byref(ms), _stream(stream)))
    return tf.value, ms.value


def mtp_get_params(model):
    out = np.zeros(model.n_params)
    _check(lib().mtp_get_params(model.h, _ptr(out), out.size))
    return out


def _refs(E_ref, F_ref, W_ref):
    E_ref = torch.as_tensor(E_ref).to(device="cuda", dtype=torch.float64).contiguous()
    F_ref = torch.as_tensor(F_ref).to(device="cuda", dtype=torch.float64).contiguous()
    if W_ref is not None:
        W_ref = torch.as_tensor(W_ref).to(device="cuda", dtype=torch.float64).contiguous()
    return E_ref, F_ref, W_ref


def mtp_fit_bfgs(model, batch, nbr, E_ref, F_ref, W_ref=None, w_e=1.0, w_f=0.01, w_s=0.0, prec="fp64",
                 max_iter=100, gtol=1e-8, stream=None):
    """BFGS fit of the model's parameters; returns (final loss, accepted steps)."""
    E_ref, F_ref, W_ref = _refs(E_ref, F_ref, W_ref)
    loss, iters = ctypes.c_double(), ctypes.c_int64()
    _check(lib().mtp_fit_bfgs(model.h, ctypes.byref(batch.c), nbr.h, _prec(prec), _ptr(E_ref), _ptr(F_ref),
                              _ptr(W_ref), float(w_e), float(w_f), float(w_s), int(max_iter), float(gtol),
                              ctypes.byref(loss), ctypes.byref(iters), _stream(stream)))
    return loss.value, iters.value


def mtp_fit_errors(model, batch, nbr, E_ref, F_ref, W_ref=None, prec="fp64", stream=None):
    """[E/atom max, mean, RMS, |dF| max, mean, RMS, |dW| max, mean, RMS]."""
    E_ref, F_ref, W_ref = _refs(E_ref, F_ref, W_ref)
    rep = np.zeros(9)
    _check(lib().mtp_fit_errors(model.h, ctypes.byref(batch.c), nbr.h, _prec(prec), _ptr(E_ref), _ptr(F_ref),
                                _ptr(W_ref), _ptr(rep), _stream(stream)))
    return rep


def mtp_profiler_enable(on=True):
    _check(lib().mtp_profiler_enable(1 if on else 0))


def mtp_profiler_read(capacity=64):
    """{region: (total_ms, launches)} since the last read (synchronises the recorded events)."""
    names = ctypes.create_string_buffer(48 * capacity)
    ms = np.zeros(capacity)
    launches = np.zeros(capacity, np.int64)
    cnt = ctypes.c_int32()
    _check(lib().mtp_profiler_read(capacity, names, _ptr(ms), _ptr(launches), ctypes.byref(cnt)))
    raw = names.raw
    out = {}
    for k in range(cnt.value):
        nm = raw[48 * k:48 * (k + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (float(ms[k]), int(launches[k]))
    return out
