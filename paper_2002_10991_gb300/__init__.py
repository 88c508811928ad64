"""GB300-native tridiagonal -> band eigenvector back-transformation
(arXiv 2002.10991, Eq. 6d), with the band -> tridiagonal reduction that feeds
it (Eq. 6b) and the band -> full back-transformation after it (Eq. 6e): a
CUDA library behind a C ABI (include/tbbt.h) and this thin Python binding."""

from .api import (  # noqa: F401
    Batch,
    bulge_chase,
    Plan,
    TbbtError,
    num_reflectors,
    release_cache,
    schedule_max_live_rows,
    stream_check,
    trans_ev_band_to_full,
    trans_ev_tridi_to_band,
    trans_ev_tridi_to_band_host,
    trans_ev_tridi_to_band_noalloc,
    tridiag_eig,
)
