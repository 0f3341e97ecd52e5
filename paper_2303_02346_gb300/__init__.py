"""GB300 (sm_103a) MLS-MPM step and reverse-mode adjoint behind a C-ABI library.

`binding` holds the ctypes functions with the C names (sim_create, sim_step,
sim_backward, ...); `simulator` adds a scene-level wrapper and the
torch.autograd.Function. The CUDA library is built in-tree by `build.build()`.
Importing this package does not load the library; the first call does, and
fails loudly if it cannot.
"""
from .binding import (SimError, make_config, sim_add_loss_grad, sim_autotune, sim_backward, sim_create,  # noqa: F401
                      sim_current_step, sim_destroy, sim_get_state, sim_grid_mass_loss, sim_kernel_launches,
                      sim_last_error, sim_position_loss, sim_profile_enable, sim_profile_read,
                      sim_set_launch, sim_set_particles, sim_set_tool, sim_step, sim_sync, sim_version)
