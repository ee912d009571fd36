"""pgc -- GB300-native speculative graph coloring (D1, D2, PD2).

The computation lives in the CUDA library ``_build/libpgc.so`` (C ABI in
``include/pgc.h``); ``binding`` marshals arguments to it.  Importing this
package does not load the library; the first call does, and fails loudly if
the library cannot be built or loaded.
"""
from .binding import (  # noqa: F401
    PGC_ASYNC, PGC_AUTOTUNE, PGC_HOST_LOOP, PGC_PRIORITY_DYNAMIC, PGC_PRIORITY_SATURATION, PGC_NO_DEGREE_RULE, PGC_VALIDATE, BatchResult, ColorResult,
    PgcError, PgcServer, Profile, RequestInfo, pgc_color_d1, pgc_color_d1_batch,
    pgc_color_d1_noalloc, pgc_color_d2, pgc_color_pd2, pgc_color_pd2_bipartite, pgc_release,
    pgc_test_core_barrier,
    pgc_test_fail_alloc, pgc_version,
)
