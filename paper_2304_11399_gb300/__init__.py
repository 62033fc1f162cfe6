"""GB300 (sm_103a) traveltime-parameter search: semblance of CMP / ZO-CRS
operators, differential evolution with Philox draws, neighbour exchange of
best individuals and adjoint-gradient polish, behind the C ABI of
include/tt.h (libtt.so, built by ``paper_2304_11399_gb300.build``)."""
from .tt import (  # noqa: F401
    TTError, Context, tt_version, tt_ctx_create, tt_ctx_load_traces, tt_semblance_eval,
    tt_semblance_grad, tt_de_step, tt_best_snapshot, tt_neighbor_exchange, tt_polish,
    tt_search, tt_ctx_profile, tt_ctx_stats, tt_ctx_set_option, tt_ctx_get_option,
    tt_ctx_autotune, tt_ens_search, tt_stack, tt_jade_state, tt_search_slab, tt_ctx_probe_l1,
    SemblanceFn,
    semblance,
)
