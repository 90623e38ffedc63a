// Pass kernels and launch shapes of the padded size M = 256.
#include "fc_variants.cuh"

namespace fc {

void variants_256(bool f64, Variants* v) {
    if (f64)
        make_variants<double, 256>(*v);
    else
        make_variants<float, 256>(*v);
}

}  // namespace fc
