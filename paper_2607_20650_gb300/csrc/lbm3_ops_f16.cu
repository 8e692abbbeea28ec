// D3Q19 kernel instantiations for storage type __half.
#include "lbm3_ops.cuh"

const Ops3 &ops3_f16() {
    static const Ops3 o = make_ops3<__half>();
    return o;
}
