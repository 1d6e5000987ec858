"""GB300-native (sm_103a) super-droplet warm-rain microphysics hot path.

The library itself is the C ABI in ``include/sdm.h`` (``_build/libsdm.so``);
``paper_1310_1905_gb300.sdm`` is its thin ctypes binding.
"""
from .sdm import (Particles, SdmError, load, sdm_destroy, sdm_diag_mom, sdm_diag_rng,  # noqa: F401
                  sdm_diag_sd_conc, sdm_get_attr, sdm_get_fields, sdm_get_stats, sdm_get_step,
                  sdm_get_timing, sdm_init, sdm_outbuf, sdm_set_attr, sdm_set_step, sdm_sizes,
                  sdm_step_async, sdm_step_sync, sdm_timing_enable, sdm_wait)
