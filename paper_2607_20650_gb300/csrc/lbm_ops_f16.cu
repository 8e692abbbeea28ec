// Kernel instantiations for storage type __half.
#include "lbm_kernels.cuh"

namespace lbm {
const Ops &ops_f16() {
    static const Ops o = make_ops<__half>();
    return o;
}
}  // namespace lbm
