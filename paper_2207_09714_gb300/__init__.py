"""GB300-native library for the per-day step of GradABM (differentiable agent-based
epidemiology): CUDA kernels for sm_103a behind the C ABI of include/gabm.h, a thin
ctypes binding with the same names (``capi``), a torch.autograd.Function
(``autograd.GabmFunction``) and seeded synthetic population generators (``synth``)."""

from .capi import (GABM_DEVICE, GABM_HOST, GABM_NEVER, GABM_RECOMPUTE, GABM_STORE_LAMBDA, GabmCtx,
                   GabmError, ModelDesc, gabm_backward, gabm_create, gabm_destroy, gabm_forward,
                   gabm_get_lambda, gabm_get_profile, gabm_get_state, gabm_launch_count, gabm_mem_stats,
                   gabm_mse_loss, gabm_philox, gabm_set_profiling, gabm_set_state, gabm_version,
                   load_library)

__all__ = [n for n in dir() if n.startswith(("gabm_", "GABM_"))] + [
    "GabmCtx", "GabmError", "ModelDesc", "load_library"]
