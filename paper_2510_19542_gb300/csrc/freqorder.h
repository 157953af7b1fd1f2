// Frequency order of the persistent frame kernel's warp transforms.
//
// A length-M transform runs in LW = min(M, 32) lanes with R = M / LW values
// per lane.  Its forward output leaves frequency j = k_r + R * brev(t) in
// register k_r of lane t, where brev reverses the log2(LW) bits of t.  B, the
// removeTT spectra and the column spectra of the kernel are stored in that
// order along j: position pos = k_r * LW + t holds frequency j.
#pragma once

#include <cuda_runtime.h>

namespace safr {

__host__ __device__ constexpr int wfft_lanes(int M) { return M < 32 ? M : 32; }

__host__ __device__ inline int bit_reverse(int x, int bits)
{
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}

__host__ __device__ inline int log2_exact(int n)
{
    int b = 0;
    while ((1 << b) < n) ++b;
    return b;
}

// frequency j held at storage position pos
__host__ __device__ inline int wfft_j_of_pos(int pos, int M)
{
    const int LW = wfft_lanes(M), R = M / LW;
    return pos / LW + R * bit_reverse(pos % LW, log2_exact(LW));
}

// storage position of frequency j
__host__ __device__ inline int wfft_pos_of_j(int j, int M)
{
    const int LW = wfft_lanes(M), R = M / LW;
    return (j % R) * LW + bit_reverse(j / R, log2_exact(LW));
}

}  // namespace safr
