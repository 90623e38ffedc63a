// Pass kernels and launch shapes of the padded size M = 512.
#include "fc_variants.cuh"

namespace fc {

void variants_512(bool f64, Variants* v) {
    if (f64)
        make_variants<double, 512>(*v);
    else
        make_variants<float, 512>(*v);
}

}  // namespace fc
