// md_fft.cuh -- the 3-D FFTs of the SPME reciprocal chain, hand-written
// (md_fft.cu): a real grid Q[z][y][x] (x fastest) of K_z x K_y x K_x and its
// half spectrum Qhat[m_z][m_y][m_x], m_x < K_x / 2 + 1, with the conventions
// of an unnormalised real-to-complex transform: forward
// Qhat(m) = sum_r Q(r) exp(-2 pi i m.r / K), inverse without the 1/N factor.
//
// The reciprocal chain runs as five passes over the grid: the x pass (real to
// half-complex rows) and the y pass of the forward transform; one z pass that
// takes each z line forward, multiplies it by the influence function theta,
// accumulates the energy sum theta |Qhat|^2 and takes it back; then the
// inverse y and x passes.  Every pass stages tiles of whole lines in shared
// memory and transforms them there with mixed-radix Stockham stages (radix
// 16, 8, 6, 4, 2, 3, 5, 7); axis lengths must factor into 2, 3, 5 and 7.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mdb {

constexpr int kFftMaxStages = 16;

struct FftAxis {
    int n = 0;                  // length
    int nst = 0;                // Stockham stages
    int rad[kFftMaxStages] = {};  // radix of each stage (product n)
    uint32_t mg[kFftMaxStages] = {};  // ceil(2^32 / Ns) of each stage (Ns > 1)
    uint32_t mn = 0;            // ceil(2^32 / n)
    int lp = 1;                 // lines per shared-memory tile (1, 2, 4, 8 or 16)
    int ls = 1;                 // line stride in the tile (lp + 1 pads against bank conflicts)
    void *tw = nullptr;         // device table exp(-2 pi i k / n), k < n, complex R
};

struct Fft3 {
    int K[3] = {0, 0, 0};       // K_x, K_y, K_z
    int Kh = 0;                 // K_x / 2 + 1
    bool f32 = true;            // R = float (else double)
    FftAxis ax[3];
};

// Radices for an axis of length n (16s first (FP64 only: in FP32 the radix-16
// butterfly's registers cost more than its saved stage), then 8, 6, 4, 2, 3,
// 5, 7); false if n has another prime factor or needs more than kFftMaxStages
// stages.
bool fft_factor(int n, bool f32, int *rad, int *nst);

// Plans the three axes (twiddle tables on the device, tile sizes); false with
// an error code on failure (cudaErrorInvalidValue: an axis that does not
// factor).  fft3_free releases the tables.
cudaError_t fft3_plan(Fft3 *p, const int K[3], bool f32);
void fft3_free(Fft3 *p);

// Forward x and y passes: grid (real) -> ghat (half spectrum).
cudaError_t fft3_forward_xy(const Fft3 &p, const void *grid, void *ghat, cudaStream_t st);
// Fused z pass over ghat, in place: forward along z, the influence multiply
// and energy partials (nparts CTAs, each writing part[k] = its share of
// sum w(m_x) theta |Qhat|^2, w = 1 for m_x = 0 and m_x = K_x / 2, else 2),
// inverse along z.
cudaError_t fft3_z_influence(const Fft3 &p, void *ghat, const void *theta, double *part,
                             int nparts, cudaStream_t st);
// Inverse y and x passes: ghat -> grid (real, unnormalised).
cudaError_t fft3_inverse_yx(const Fft3 &p, void *ghat, void *grid, cudaStream_t st);

}  // namespace mdb
