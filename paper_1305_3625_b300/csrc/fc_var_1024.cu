// Pass kernels and launch shapes of the padded size M = 1024.
#include "fc_variants.cuh"

namespace fc {

void variants_1024(bool f64, Variants* v) {
    if (f64)
        make_variants<double, 1024>(*v);
    else
        make_variants<float, 1024>(*v);
}

}  // namespace fc
