"""GB300-native BatMap all-pairs support counting (Amossen & Pagh, IPDPS 2011).

The compute path is the CUDA library libbatmap.so (include/batmap.h); this
package holds its sources (csrc/), the build step (_build.py) and the Python
binding (batmap.py).  Importing the binding's functions requires the built
library; there is no CPU fallback.
"""
from .batmap import (  # noqa: F401
    BATMAP_ERR_ARG, BATMAP_ERR_CAPACITY, BATMAP_ERR_CUDA, BATMAP_ERR_INTERNAL, BATMAP_ERR_NOMEM,
    BATMAP_ERR_TIMEOUT, BATMAP_OK, NUM_SHAPES, BatmapError, BatMapSet, batmap_build, batmap_default_params,
    batmap_export_layout, batmap_free, batmap_get_info, batmap_get_timing, batmap_kernel_launches,
    load_library, pair_support_all,
    pair_support_batch, pair_support_dense, pair_support_host, pair_threshold_noalloc,
    BatMapPool, batmap_pool_create, batmap_pool_free, batmap_pool_info, intersect_query, batmap_serve,
    batmap_serve_opts, batmap_autotune, batmap_release_scratch, intersect_query_list, batmap_build_cross,
    batmap_build_d, itemset_support, frequent_triples, batmap_test_dense_timeout,
    frequent_quadruples,
)
