"""GB300-native thin-nanodisk micromagnetics (Wysin & Figueiredo 2012).

The computation lives in the CUDA library libnanodisk.so behind the C ABI of
``include/nanodisk.h``; this package is its Python binding.  ``Nanodisk``
wraps one handle and marshals states between the library's flat
[replica][3][D][Dpad] layout and per-replica (3, D, D) grids.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import _binding as _b
from ._binding import (ND_METHOD_HEUN, ND_METHOD_RK4, nd_autotune, nd_autotune_group, nd_plan_info, nd_set_plan, nd_graph_create, nd_graph_destroy, nd_graph_launch,
                       nd_graph_join,
                       nd_graph_nodes, nd_check_status, nd_selftest_handover_timeout, nd_series_reset,
                       nd_series_sample, nd_series_read, nd_power_spectrum, ND_GRAPH_STATS, ND_GRAPH_SERIES, ND_ERR_ARG, ND_ERR_CUDA, ND_ERR_NAN, ND_ERR_NO_VORTEX, ND_ERR_NOT_CONVERGED, ND_ERR_TIMEOUT,
                       ND_FP32, ND_FP64, ND_GRID_3X, ND_OK, NDError, nd_create_disk, nd_destroy, nd_disk_desc, nd_disk_mask,
                       nd_effective_field, nd_energy, nd_get_info, nd_init_vortex, nd_last_error, nd_mean_m,
                       nd_relax_constrained, nd_replica_layout, nd_set_damping, nd_set_green_tensor, nd_step_heun,
                       nd_set_mask, nd_set_field_schedule,
                       nd_stats_read, nd_stats_reset, nd_stats_sample, nd_stats_save, nd_stats_load, nd_step_rk4, nd_units,
                       nd_vortex_core)

__all__ = ["Disk", "Nanodisk", "NDError", "ND_FP32", "ND_FP64", "ND_GRID_3X", "nd_create_disk", "nd_destroy", "nd_effective_field",
           "nd_energy", "nd_step_rk4", "nd_step_heun", "nd_init_vortex", "nd_vortex_core", "nd_mean_m",
           "nd_set_green_tensor", "nd_set_damping", "nd_set_mask", "nd_set_field_schedule", "nd_units", "nd_replica_layout", "nd_get_info",
           "nd_disk_mask", "nd_last_error", "nd_relax_constrained",
           "nd_stats_reset", "nd_stats_sample", "nd_stats_read", "nd_stats_save", "nd_stats_load", "nd_check_status", "nd_selftest_handover_timeout",
           "nd_series_reset", "nd_series_sample", "nd_series_read", "nd_power_spectrum", "ND_GRAPH_STATS", "ND_GRAPH_SERIES",
           "nd_graph_create", "nd_graph_launch", "nd_graph_join", "nd_graph_nodes", "nd_graph_destroy",
           "nd_autotune", "nd_autotune_group", "nd_plan_info", "nd_set_plan"]


@dataclass
class Disk:
    """Geometry and material of one disk (SI units)."""
    R: float
    L: float
    a: float = 2e-9
    Ms: float = 8.6e5
    A: float = 1.3e-11
    gamma: float = 1.76e11
    alpha: float = 0.0
    hext: tuple = (0.0, 0.0, 0.0)
    polarity: int = 1
    chirality: int = 1

    def desc(self) -> nd_disk_desc:
        return nd_disk_desc(self.R, self.L, self.a, self.Ms, self.A, self.gamma, self.alpha,
                            (ctypes_double3(*self.hext)), int(self.polarity), int(self.chirality))


def ctypes_double3(*v):
    import ctypes
    return (ctypes.c_double * 3)(*v)


class Nanodisk:
    """One library handle: disks, replicas and their state layout."""

    def __init__(self, disks, replicas=None, precision=ND_FP32, grid3x=False):
        """grid3x: allow the padded sizes 192 (3 x 64) for disks of 65..96 cells
        and 200 (8 x 25) for disks of 97..100 cells."""
        disks = list(disks) if isinstance(disks, (list, tuple)) else [disks]
        self.disks = disks
        self.precision = precision
        self.h = nd_create_disk([d.desc() for d in disks], replicas, precision | (ND_GRID_3X if grid3x else 0))
        self.B, self.state_elems = nd_get_info(self.h)
        self.layout = [nd_replica_layout(self.h, r) for r in range(self.B)]
        self.rep_disk = []
        for d, n in enumerate(replicas if replicas is not None else [1] * len(disks)):
            self.rep_disk += [d] * n
        self.units = [nd_units(self.h, d) for d in range(len(disks))]
        self.dtype = np.float64 if precision == ND_FP64 else np.float32

    def close(self):
        if getattr(self, "h", None):
            nd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------- marshalling
    def pack(self, grids) -> np.ndarray:
        """Per-replica (3, D, D) arrays -> flat host state buffer."""
        out = np.zeros(self.state_elems, dtype=self.dtype)
        for r, g in enumerate(grids):
            L = self.layout[r]
            D, Dp, off = L["D"], L["Dpad"], L["offset"]
            blk = np.zeros((3, D, Dp), dtype=self.dtype)
            blk[:, :, :D] = g
            out[off:off + 3 * D * Dp] = blk.ravel()
        return out

    def unpack(self, flat) -> list:
        """Flat state buffer (numpy or torch) -> list of (3, D, D) float64 arrays."""
        if hasattr(flat, "detach"):
            flat = flat.detach().cpu().numpy()
        res = []
        for r in range(self.B):
            L = self.layout[r]
            D, Dp, off = L["D"], L["Dpad"], L["offset"]
            res.append(np.asarray(flat[off:off + 3 * D * Dp], dtype=np.float64).reshape(3, D, Dp)[:, :, :D].copy())
        return res

    def empty_device(self):
        import torch
        return torch.zeros(self.state_elems, dtype=torch.float64 if self.precision == ND_FP64 else torch.float32,
                           device="cuda")

    def to_device(self, grids):
        import torch
        return torch.from_numpy(self.pack(grids)).cuda()

    def mask(self, d=0):
        D = self.layout[self.rep_disk.index(d)]["D"]
        return nd_disk_mask(self.h, d, D)

    # ------------------------------------------------------------- calls
    def field(self, m, b=None, stream=None):
        if b is None:
            b = self.empty_device() if hasattr(m, "data_ptr") else np.zeros_like(m)
        nd_effective_field(self.h, m, b, stream)
        return b

    def energy(self, m, stream=None):
        return nd_energy(self.h, m, self.B, stream)

    def rk4(self, m, n_steps, dt_seconds, stream=None):
        nd_step_rk4(self.h, m, n_steps, dt_seconds, stream)
        return m

    def heun(self, m, n_steps, dt_seconds, T_kelvin, seed, step0=0, stream=None):
        nd_step_heun(self.h, m, n_steps, dt_seconds, T_kelvin, seed, step0, stream)
        return m

    def init_vortex(self, m, X0, stream=None):
        nd_init_vortex(self.h, m, np.asarray(X0, dtype=np.float64).reshape(self.B, 2), stream)
        return m

    def vortex_core(self, m, stream=None):
        return nd_vortex_core(self.h, m, self.B, stream)

    def relax(self, m, X, tol=1e-6, max_iter=20000, stream=None):
        """Constrained relaxation in place; returns (status, U, lambda, iters)."""
        return nd_relax_constrained(self.h, m, np.asarray(X, dtype=np.float64).reshape(self.B, 2), self.B, tol,
                                    max_iter, stream)

    def mean_m(self, m, stream=None):
        return nd_mean_m(self.h, m, self.B, stream)

    def set_damping(self, alpha):
        nd_set_damping(self.h, np.broadcast_to(np.asarray(alpha, dtype=np.float64), (self.B,)).copy())

    def set_green_tensor(self, d, Gq=None):
        nd_set_green_tensor(self.h, d, Gq)

    def set_mask(self, d, mask):
        """Replace disk d's mask by any cell set of its grid (refreshes the layout)."""
        nd_set_mask(self.h, d, mask)
        self.layout = [nd_replica_layout(self.h, r) for r in range(self.B)]
        self.units = [nd_units(self.h, k) for k in range(len(self.disks))]

    def set_field_schedule(self, d, H=None):
        """Per-step external field H[s] in A/m, shape (n, 3); None removes it."""
        nd_set_field_schedule(self.h, d, H)

    def dtau(self, dt_seconds, d=0):
        return dt_seconds / self.units[d][3]
