"""GB300-native PRNGD: extended-precision uniform variates (Demchik and Gulov, arXiv:1401.8230).

Thin ctypes binding over ``libprngd.so`` (C ABI in ``include/prngd.h``). Every function here
only marshals arguments: device memory and CUDA streams come from PyTorch tensors / streams
(or raw integer pointers), and all generation runs in the library's CUDA kernels. There is no
CPU fallback: if the library is missing or cannot be built, the calls raise.
"""
from ._binding import (  # noqa: F401
    FORM_A_FP64,
    FORM_B_INTBITS,
    FORM_C_F32PAIR,
    PRNG_EBUSY,
    PRNG_ECUDA,
    PRNG_EINVAL,
    PRNG_ENOMEM,
    PRNG_ENOTFOUND,
    PRNG_ETIMEOUT,
    PRNG_OK,
    Generator,
    MAX_BATCH_REQUESTS,
    REQ_FRESH,
    REQ_RESIDENT,
    PrngError,
    Request,
    fresh_request,
    lib,
    prng_batch_get_shape,
    prng_batch_set_shape,
    prng_create,
    prng_destroy,
    prng_fill_f32pair,
    prng_fill_f64,
    prng_fill_f64_host,
    prng_fill_f64_host_noalloc,
    prng_fused_stats,
    prng_get_info,
    prng_last_error,
    prng_poll,
    prng_state_bytes,
    prng_state_restore,
    prng_state_save,
    prng_submit,
    prng_version,
    prng_wait,
    resident_request,
)
