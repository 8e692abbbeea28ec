// Kernel instantiations for storage type __nv_bfloat16.
#include "lbm_kernels.cuh"

namespace lbm {
const Ops &ops_bf16() {
    static const Ops o = make_ops<__nv_bfloat16>();
    return o;
}
}  // namespace lbm
