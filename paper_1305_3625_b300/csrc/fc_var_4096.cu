// Pass kernels and launch shapes of the padded size M = 4096.
#include "fc_variants.cuh"

namespace fc {

void variants_4096(bool f64, Variants* v) {
    if (f64)
        make_variants<double, 4096>(*v);
    else
        make_variants<float, 4096>(*v);
}

}  // namespace fc
