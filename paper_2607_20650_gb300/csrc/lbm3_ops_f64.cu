// D3Q19 kernel instantiations for storage type double.
#include "lbm3_ops.cuh"

const Ops3 &ops3_f64() {
    static const Ops3 o = make_ops3<double>();
    return o;
}
