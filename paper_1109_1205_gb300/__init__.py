"""GB300 (sm_103a) Krylov-space Green's-function solver: Python binding.

The binding only marshals arguments to libkrylovgf (include/krylovgf.h);
every numerical step runs in the library's CUDA kernels.  The functions keep
the C names (kg_build_sector, kg_hpsi, ...); `Sector` and `Keldysh` wrap the
handles for convenience.  Importing this package loads the compiled library
and raises ImportError if it has not been built -- there is no CPU fallback.
"""
from __future__ import annotations

from ._lib import (  # noqa: F401
    KG_OK, KG_EINVAL, KG_ENOMEM, KG_ENOCONV, KG_EDEGEN, KG_EBREAKDOWN, KG_ENUMERIC, KG_ETIMEOUT,
    KG_ECUDA, KGError, Opts, Sector, Keldysh, lib, library_path, kg_opts_default, kg_build_sector,
    kg_free_sector, kg_sector_dims, kg_sector_strings, kg_hpsi, kg_neighbour_dim, kg_apply_cop,
    kg_ground_state, kg_copy_ground_state, kg_propagate, kg_green_equilibrium, kg_green_keldysh,
    kg_keldysh_create, kg_keldysh_row, kg_keldysh_gram, kg_keldysh_get_phi, kg_keldysh_set_phi,
    kg_keldysh_free, kg_keldysh_plan, kg_strerror, kg_last_error, kg_launch_count, kg_profile_start, kg_profile_stop,
    kg_probe_fp64, kg_overlaps, kg_green_equilibrium_batched, kg_green_equilibrium_vjp, kg_green_lanczos,
    kg_green_equilibrium_fine, kg_green_fourier, kg_overlaps_noalloc, kg_green_matsubara,
    kg_green_matsubara_steps, kg_green_mixed, kg_green_restarted, kg_green_keldysh_td, kg_keldysh_create_td,
    kg_green_four_time, kg_necpt_occupations,
)
