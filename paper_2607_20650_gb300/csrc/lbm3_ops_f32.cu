// D3Q19 kernel instantiations for storage type float.
#include "lbm3_ops.cuh"

const Ops3 &ops3_f32() {
    static const Ops3 o = make_ops3<float>();
    return o;
}
