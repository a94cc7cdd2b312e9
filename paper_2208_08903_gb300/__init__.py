"""GB300 (sm_103a) flow-based sampler for lattice phi^4 theory.

Hot path (arXiv:2208.08903): prior -> checkerboard RealNVP coupling stack ->
log q, phi^4 action, log w -> Metropolis-Hastings independence chain, plus the
reverse-KL training step and the FP64 HMC comparison sampler.  The CUDA
library libgfflow.so (C ABI: include/gfflow.h) does all the arithmetic; this
package is its ctypes/torch binding.
"""
from .api import (Flow, SampleResult, autocorr, chain_gather, device_status, ess,  # noqa: F401
                  hmc_trajectory, mh_chain, observables,
                  mh_chain_noalloc,
                  mh_chain_workspace_bytes, new_mh_state, phi4_action, phi4_action_vjp,
                  phi4_force, read_mh_state, set_stream_status_slot, tensor_core_supported)
from . import autograd  # noqa: F401
