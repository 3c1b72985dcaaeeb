"""GB300 (sm_103a) preconditioned block BiCGGR for the clover Wilson-Dirac equation (arXiv:0907.3261).

The compute path is the CUDA library ``libbbicggr.so`` (sources in ``csrc/``, C-ABI in
``include/bbicggr.h``); ``_lib`` is its ctypes binding with the same entry-point names.
``inputs`` holds the seeded synthetic input generators.
"""
from ._lib import (Net, bbicggr_solve_batch, wd_net_adam_step, wd_net_apply, wd_net_create, wd_net_destroy,
                   wd_net_get_weights, wd_net_loss_grad, wd_net_set_weights)
from ._lib import (WD_BREAKDOWN, WD_DIVERGED, WD_LMAX, WD_NOT_CONVERGED, WD_OK, Context, WDError,
                   jacobi_precond_noalloc, bb_update_u, bb_update_xr, bb_update_pv, wd_set_domain,
                   bbicggr_solve, jacobi_precond, wd_apply, wd_create, wd_destroy,
                   wd_profile_enable, wd_profile_read, wd_profile_reset, wd_set_tile, wd_tuned_tile,
                   wd_link_reals, wd_set_link_reals, wd_set_apply_form,
                   wd_get_apply_form, wd_copy_residual)

__all__ = ["Net", "bbicggr_solve_batch", "wd_net_create", "wd_net_destroy", "wd_net_apply", "wd_net_loss_grad",
           "wd_net_adam_step", "wd_net_get_weights", "wd_net_set_weights", "wd_create", "wd_destroy", "wd_apply", "jacobi_precond", "bbicggr_solve", "Context",
           "WDError", "wd_profile_enable", "wd_profile_read", "wd_profile_reset", "WD_OK", "WD_NOT_CONVERGED", "WD_DIVERGED", "WD_BREAKDOWN", "WD_LMAX",
           "wd_set_tile", "wd_tuned_tile", "wd_link_reals", "wd_set_link_reals", "wd_set_apply_form", "wd_get_apply_form", "wd_copy_residual", "jacobi_precond_noalloc",
           "bb_update_u", "bb_update_xr", "bb_update_pv", "wd_set_domain"]
