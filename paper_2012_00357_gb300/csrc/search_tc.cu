// Tensor-core exact search: placeholder until the tcgen05 kernel lands.
#include "dd_internal.cuh"

dd_status dd_build_fp16(dd_dataset *ds) {
    return dd_fail(ds->ctx, DD_ERR_STATE, "tensor-core search not built yet");
}

dd_status dd_search_exact_tc(dd_dataset *ds, const double *, int64_t, int, SearchOut, dd_search_stats *,
                             cudaStream_t) {
    return dd_fail(ds->ctx, DD_ERR_STATE, "tensor-core search not built yet");
}
