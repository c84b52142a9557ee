// Table block of the column-pruned fused kernel (k_fused128p) for one polarisation: layout shared by the host
// builder (plan.cpp, FP64 arithmetic stored FP32) and the kernel, which copies the block to shared memory once.
//
// The kernel transforms along x first (row pairs packed as one complex row), keeps only the columns k_x of the
// box that the circular window touches (the set K = [kxlo, kxlo + nk), contiguous), and runs the y transform,
// the window selection and the y inverse once per kept column.  Columns outside K are zero after the window
// and are never transformed along y.
#pragma once

namespace dhk {

constexpr int kPrN = 128;        // window size
constexpr int kPrM = 64;         // field size
constexpr int kPrMaxK = 48;      // most kept columns (the guide's radius rule gives at most 42 at N = 128)
constexpr int kPrG = 16;         // most HG groups

// Byte offsets inside the block (every table starts on a 16-byte boundary).
struct PrLayout {
    static constexpr int HDR = 0;                         // int[16]: nk, kxlo, klx, kly
    static constexpr int QLIM = 64;                       // int2[kPrMaxK]: kept box rows [qlo, qhi] of column c
    static constexpr int PHX = QLIM + 8 * kPrMaxK;        // float2[kPrMaxK]: x beam-centre phase of column c, x 1/2
    static constexpr int PHY = PHX + 8 * kPrMaxK;         // float2[M]: y beam-centre phase of box row q
    static constexpr int CY = PHY + 8 * kPrM;             // float2[M]: y residual tilt and defocus removal
    static constexpr int CX = CY + 8 * kPrM;              // float2[M]: x residual tilt and defocus removal
    static constexpr int TWN = CX + 8 * kPrM;             // float2[N]: exp(-2 pi i k / N), the twiddle bases
    static constexpr int HGY = TWN + 8 * kPrN;            // float[M][20]: u_n(y'_j) dy' at [j][n] (n < 16)
    static constexpr int V = HGY + 4 * kPrM * 20;         // float2[16][kPrMaxK]: x contraction of column c
    static constexpr int BYTES = V + 8 * kPrG * kPrMaxK;
};

}  // namespace dhk
