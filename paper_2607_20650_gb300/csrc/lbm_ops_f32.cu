// Kernel instantiations for storage type float.
#include "lbm_kernels.cuh"

namespace lbm {
const Ops &ops_f32() {
    static const Ops o = make_ops<float>();
    return o;
}
}  // namespace lbm
