// Pass kernels and launch shapes of the padded size M = 8192.
#include "fc_variants.cuh"

namespace fc {

void variants_8192(bool f64, Variants* v) {
    if (f64)
        make_variants<double, 8192>(*v);
    else
        make_variants<float, 8192>(*v);
}

}  // namespace fc
