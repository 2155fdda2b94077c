// Approximate search: placeholder until the k-means partition lands.
#include "dd_internal.cuh"

dd_status dd_build_ann(dd_dataset *ds, const dd_dataset_opts &) {
    return dd_fail(ds->ctx, DD_ERR_STATE, "ANN search not built yet");
}

dd_status dd_search_ann(dd_dataset *ds, const double *, int64_t, double, const int32_t *, SearchOut,
                        dd_search_stats *, cudaStream_t) {
    return dd_fail(ds->ctx, DD_ERR_STATE, "ANN search not built yet");
}

void dd_free_ann(dd_dataset *) {}
