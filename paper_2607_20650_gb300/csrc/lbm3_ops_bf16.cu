// D3Q19 kernel instantiations for storage type __nv_bfloat16.
#include "lbm3_ops.cuh"

const Ops3 &ops3_bf16() {
    static const Ops3 o = make_ops3<__nv_bfloat16>();
    return o;
}
