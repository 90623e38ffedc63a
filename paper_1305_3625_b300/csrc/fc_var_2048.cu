// Pass kernels and launch shapes of the padded size M = 2048.
#include "fc_variants.cuh"

namespace fc {

void variants_2048(bool f64, Variants* v) {
    if (f64)
        make_variants<double, 2048>(*v);
    else
        make_variants<float, 2048>(*v);
}

}  // namespace fc
