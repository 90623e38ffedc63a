// Pass kernels and launch shapes of the padded sizes M = 2 .. 128.
#include "fc_variants.cuh"

namespace fc {

template <typename T>
static bool small_t(int M, Variants* v) {
    switch (M) {
        case 2: make_variants<T, 2>(*v); return true;
        case 4: make_variants<T, 4>(*v); return true;
        case 8: make_variants<T, 8>(*v); return true;
        case 16: make_variants<T, 16>(*v); return true;
        case 32: make_variants<T, 32>(*v); return true;
        case 64: make_variants<T, 64>(*v); return true;
        case 128: make_variants<T, 128>(*v); return true;
        default: return false;
    }
}

bool variants_small(int M, bool f64, Variants* v) { return f64 ? small_t<double>(M, v) : small_t<float>(M, v); }

}  // namespace fc
