// Mixed-precision tensor-core path (placeholder until the tcgen05 kernels land):
// every entry fails loudly instead of computing anything elsewhere.
#include "lattice_sum.h"
#include "ls_tc.cuh"

namespace ls {

int tc_core(const double*, const double*, const double*, const int32_t*, const int32_t*, const int32_t*,
            const double*, int64_t, double*, int, cudaStream_t, std::string* err) {
    if (err) *err = "LS_MIXED core contraction is not built in this library";
    return LS_ERR_ARG;
}

int tc_eval(const double* const*, const int32_t*, const double*, int64_t, const int32_t*, int, double*, void*,
            int, int, cudaStream_t, std::string* err) {
    if (err) *err = "LS_MIXED slab evaluation is not built in this library";
    return LS_ERR_ARG;
}

}  // namespace ls
