// Kernel instantiations for storage type double.
#include "lbm_kernels.cuh"

namespace lbm {
const Ops &ops_f64() {
    static const Ops o = make_ops<double>();
    return o;
}
}  // namespace lbm
