// Block-CSR row routine shared by the kernels that apply a generic
// block-CSR operator (the generic matrix the paper's solver takes, Sec. 3):
// the matrix is held in sliced ELL, 32 block rows per slice, block k of every
// row of a slice stored lane-interleaved ([slot][component][lane]).
#pragma once
#include "engine.h"

namespace msc {

template <class T> using T2 = typename C2<T>::t;

// y = A src for one row (thread = row, lanes of a warp = rows of a slice).
// Slice bases are 64-bit; offsets inside a slice (k * 32 * BD * BD) stay
// 32-bit; the source gathers go through the read-only path.
template <class T, int BD>
__device__ __forceinline__ void bsr_row(const OpDev& A, const T2<T>* __restrict__ vals,
                                        const T2<T>* __restrict__ src, int row, T2<T> (&y)[BD]) {
    const int slice = row >> 5;
    const int lane = row & 31;
    const int len = __ldg(&A.slice_len[slice]);
    const int64_t st = __ldg(&A.slice_start[slice]);
#pragma unroll
    for (int a = 0; a < BD; ++a) y[a] = {T(0), T(0)};
    const int32_t* __restrict__ cp = A.cols + st * 32 + lane;
    const T2<T>* __restrict__ vp = vals + st * BD * BD * 32 + lane;
#pragma unroll 3
    for (int k = 0; k < len; ++k) {
        const int c = __ldg(cp + k * 32);
        T2<T> xv[BD];
#pragma unroll
        for (int b = 0; b < BD; ++b) xv[b] = __ldg(src + (size_t)c * BD + b);
        const T2<T>* vk = vp + k * (BD * BD * 32);
#pragma unroll
        for (int a = 0; a < BD; ++a)
#pragma unroll
            for (int b = 0; b < BD; ++b) cfma(y[a], __ldg(vk + (a * BD + b) * 32), xv[b]);
    }
}

}  // namespace msc
