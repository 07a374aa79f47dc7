// The out-of-place batch kernels (one per store class of `out` relative to
// `in`, chunk width and vector width), compiled apart from the other forms
// so that the two translation units build in parallel.
#include "batch.cuh"

namespace u16wf {

const void *batch_out_kernel(int st, int nw, int vb, bool pf) {
    switch (st) {
        case 32: return words_kernel_ptr<kModeOut, 32>(nw, vb, pf);
        case 16: return words_kernel_ptr<kModeOut, 16>(nw, vb, pf);
        case 8: return words_kernel_ptr<kModeOut, 8>(nw, vb, pf);
        case 4: return words_kernel_ptr<kModeOut, 4>(nw, vb, pf);
        default: return words_kernel_ptr<kModeOut, 2>(nw, vb, pf);
    }
}

}  // namespace u16wf
