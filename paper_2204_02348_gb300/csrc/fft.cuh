// Device building blocks for batched mixed-radix FFTs on shared-memory tiles.
//
// A tile holds nb independent transforms of length L; element e of transform b sits at buf[e * es + b], so
// consecutive threads work on consecutive transforms and every pass reads and writes shared memory without
// bank conflicts (es is the padded row pitch).  Forward transforms are decimation-in-frequency (natural
// order in, digit-reversed order out); inverse transforms are decimation-in-time (digit-reversed order in,
// natural order out).  The digit-reversed positions come from a host-built table pos[k], so the gathers
// that sit between transforms (window selection, spectrum extraction, scratch loads) absorb the
// reordering.  Twiddles come from tables built on the host in FP64 and stored in FP32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dhk {

// Complex sums as one packed two-lane FP32 addition (round to nearest in each lane, as two scalar additions).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward sign) or +i (inverse sign)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ---------------------------------------------------------------------------------------------- butterflies
// y_k = sum_r a_r exp(-+ 2 pi i r k / R), in place.  Constants are exact values of cos/sin of multiples of
// pi/8 and pi/3 written to float precision.

template <bool INV>
__device__ __forceinline__ void dft2(float2* a) {
    const float2 t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_mi<INV>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2* a) { dft4<INV>(a[0], a[1], a[2], a[3]); }

constexpr float kC8 = 0.70710678118654752440f;  // cos(pi/4)

template <bool INV>
__device__ __forceinline__ float2 w8(int k, float2 v) {
    // v * exp(-+ 2 pi i k / 8) for k = 0..3
    const float sg = INV ? 1.0f : -1.0f;
    switch (k) {
        case 0: return v;
        case 1: return cmul(v, make_float2(kC8, sg * kC8));
        case 2: return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
        default: return cmul(v, make_float2(-kC8, sg * kC8));
    }
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* a) {
    float2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    float2 o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    o1 = w8<INV>(1, o1);
    o2 = w8<INV>(2, o2);
    o3 = w8<INV>(3, o3);
    a[0] = cadd(e0, o0); a[4] = csub(e0, o0);
    a[1] = cadd(e1, o1); a[5] = csub(e1, o1);
    a[2] = cadd(e2, o2); a[6] = csub(e2, o2);
    a[3] = cadd(e3, o3); a[7] = csub(e3, o3);
}

template <bool INV>
__device__ __forceinline__ void dft16(float2* a) {
    float2 e[8], o[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { e[i] = a[2 * i]; o[i] = a[2 * i + 1]; }
    dft8<INV>(e);
    dft8<INV>(o);
    // cos(k pi / 8), sin(k pi / 8), k = 0..7
    const float c[8] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508978f,
                        0.0f, -0.38268343236508978f, -0.70710678118654752f, -0.92387953251128674f};
    const float s[8] = {0.0f, 0.38268343236508978f, 0.70710678118654752f, 0.92387953251128674f,
                        1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508978f};
    const float sg = INV ? 1.0f : -1.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        // k = 4 is a quarter turn: an exact swap and negation, no multiplication
        const float2 t = (k == 0) ? o[k] : (k == 4) ? mul_mi<INV>(o[k]) : cmul(o[k], make_float2(c[k], sg * s[k]));
        a[k] = cadd(e[k], t);
        a[k + 8] = csub(e[k], t);
    }
}

template <bool INV>
__device__ __forceinline__ void dft3(float2* a) {
    const float h = 0.86602540378443865f;  // sqrt(3)/2
    const float2 s = cadd(a[1], a[2]);
    const float2 t = make_float2(a[0].x - 0.5f * s.x, a[0].y - 0.5f * s.y);
    const float2 d = mul_mi<INV>(cscale(csub(a[1], a[2]), h));
    a[0] = cadd(a[0], s);
    a[1] = cadd(t, d);
    a[2] = csub(t, d);
}

// R-point DFT for an odd prime R with roots of unity from the transform's own twiddle table (tw[e * step] is
// the R-th root W raised to e, for e in [0, R)).  Used for the odd primes 5..19 of reduced field sizes.
// Inputs r and R - r meet conjugate roots, W^{(R-r)k} = conj(W^{rk}), so with s_r = a_r + a_{R-r} and
// d_r = a_r - a_{R-r}:  y_k = a_0 + sum_r s_r Re(W^{rk}) + i d_r Im(W^{rk}) and y_{R-k} the same with the
// second sum negated (r, k = 1 .. (R-1)/2): a quarter of the multiplications of the plain sum.
template <int R>
__device__ __forceinline__ void dft_direct(float2* a, const float2* __restrict__ tw, int step) {
    static_assert(R % 2 == 1, "odd radix");
    constexpr int H = (R - 1) / 2;
    float2 sp[H], dm[H];
    float2 y0 = a[0];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
        sp[r - 1] = cadd(a[r], a[R - r]);
        dm[r - 1] = csub(a[r], a[R - r]);
        y0 = cadd(y0, sp[r - 1]);
    }
    float2 y[R];
    y[0] = y0;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        float2 ac = a[0], bc = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 1; r <= H; ++r) {
            const float2 w = tw[((r * k) % R) * step];
            ac.x = fmaf(sp[r - 1].x, w.x, ac.x);
            ac.y = fmaf(sp[r - 1].y, w.x, ac.y);
            bc.x = fmaf(-dm[r - 1].y, w.y, bc.x);
            bc.y = fmaf(dm[r - 1].x, w.y, bc.y);
        }
        y[k] = cadd(ac, bc);
        y[R - k] = csub(ac, bc);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) a[k] = y[k];
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* a, const float2* __restrict__ tw, int step) {
    if constexpr (R == 2) dft2<INV>(a);
    else if constexpr (R == 3) dft3<INV>(a);
    else if constexpr (R == 4) dft4<INV>(a);
    else if constexpr (R == 8) dft8<INV>(a);
    else if constexpr (R == 16) dft16<INV>(a);
    else dft_direct<R>(a, tw, step);
}

// ---------------------------------------------------------------------------------------------- passes
// One in-place radix-R pass of a length-L transform over nb = 2^lognb transforms.
//  DIF (INV = false): span = current block length, s = span / R; outputs twiddled by W_span^(j r).
//  DIT (INV = true) : span = block length after the pass, s = span / R; inputs twiddled by W_span^(j r).
// tw holds W_L^e for e in [0, L) with the transform's sign.
template <int R, bool INV>
__device__ __forceinline__ void fft_pass(float2* buf, int L, int span, int lognb, int es,
                                         const float2* __restrict__ tw, int tid, int nthr) {
    const int s = span / R;
    const int tw_step = L / span;
    const int nb = 1 << lognb;
    const int total = (L / R) << lognb;
    for (int t = tid; t < total; t += nthr) {
        const int b = t & (nb - 1);
        const int bf = t >> lognb;
        const int blk = bf / s;
        const int j = bf - blk * s;
        const int base = blk * span + j;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = buf[(base + r * s) * es + b];
        if (INV) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[j * r * tw_step]);
        }
        dft<R, INV>(v, tw, L / R);
        if (!INV) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[j * r * tw_step]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) buf[(base + r * s) * es + b] = v[r];
    }
}

template <bool INV>
__device__ __forceinline__ void fft_pass_any(int R, float2* buf, int L, int span, int lognb, int es,
                                             const float2* __restrict__ tw, int tid, int nthr) {
    switch (R) {
        case 2: fft_pass<2, INV>(buf, L, span, lognb, es, tw, tid, nthr); break;
        case 3: fft_pass<3, INV>(buf, L, span, lognb, es, tw, tid, nthr); break;
        case 4: fft_pass<4, INV>(buf, L, span, lognb, es, tw, tid, nthr); break;
        case 5: fft_pass<5, INV>(buf, L, span, lognb, es, tw, tid, nthr); break;
        case 7: fft_pass<7, INV>(buf, L, span, lognb, es, tw, tid, nthr); break;
        case 8: fft_pass<8, INV>(buf, L, span, lognb, es, tw, tid, nthr); break;
        case 11: fft_pass<11, INV>(buf, L, span, lognb, es, tw, tid, nthr); break;
        case 13: fft_pass<13, INV>(buf, L, span, lognb, es, tw, tid, nthr); break;
        case 16: fft_pass<16, INV>(buf, L, span, lognb, es, tw, tid, nthr); break;
        case 17: fft_pass<17, INV>(buf, L, span, lognb, es, tw, tid, nthr); break;
        case 19: fft_pass<19, INV>(buf, L, span, lognb, es, tw, tid, nthr); break;
        default: break;
    }
}

// Whole transform: radices[0..nrad) in DIF order.  Ends with a barrier.
template <bool INV>
__device__ __forceinline__ void fft_run(float2* buf, int L, const int* radices, int nrad, int lognb, int es,
                                        const float2* __restrict__ tw, int tid, int nthr) {
    if (!INV) {
        int span = L;
        for (int p = 0; p < nrad; ++p) {
            const int R = radices[p];
            fft_pass_any<false>(R, buf, L, span, lognb, es, tw, tid, nthr);
            span /= R;
            __syncthreads();
        }
    } else {
        int span = 1;
        for (int p = nrad - 1; p >= 0; --p) {
            const int R = radices[p];
            span *= R;
            fft_pass_any<true>(R, buf, L, span, lognb, es, tw, tid, nthr);
            __syncthreads();
        }
    }
}

}  // namespace dhk

namespace dhk {

// ---------------------------------------------------------------------------------------------- static passes
// Compile-time variant of one radix-R pass: NB transforms of length L, element e of transform b at
// buf[e * ES + b * BS]; DIT selects decimation in time (twiddle before the butterfly), otherwise decimation in
// frequency (twiddle after).  SPAN is the block length (DIF: before the pass; DIT: after).  tw holds W_L^k
// with the transform's sign.  Tasks are spread over NTHR threads with the transform index fastest.
template <int R, bool INV, bool DIT, int L, int SPAN, int NB, int ES, int BS, int NTHR>
__device__ __forceinline__ void spass(float2* buf, const float2* tw, int tid) {
    constexpr int S = SPAN / R;
    constexpr int TW = L / SPAN;
    constexpr int TASKS = NB * (L / R);
    for (int t = tid; t < TASKS; t += NTHR) {
        const int b = t % NB;
        const int bf = t / NB;
        const int blk = bf / S;
        const int j = bf - blk * S;
        const int base = blk * SPAN + j;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = buf[(base + r * S) * ES + b * BS];
        // with S = 1 every j is 0 and the twiddles are exactly 1
        constexpr bool TWID = S > 1;
        if (DIT && TWID) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[j * r * TW]);
        }
        dft<R, INV>(v, tw, L / R);
        if (!DIT && TWID) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[j * r * TW]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) buf[(base + r * S) * ES + b * BS] = v[r];
    }
}


// Position of index k after DIF passes of radices R0 R1 R2 (in that order; R2 = 1 for two passes): the digits
// of k, least significant first, weighted by the block lengths R1 R2, R2, 1.  The same map as the host's
// position tables, for plans fixed at compile time.
template <int R0, int R1, int R2>
__device__ __forceinline__ int dif_pos(int k) {
    return (k % R0) * (R1 * R2) + ((k / R0) % R1) * R2 + k / (R0 * R1);
}

// Position of index k: from the host's table for a runtime plan (R0 = 0), else computed.
template <int R0, int R1, int R2>
__device__ __forceinline__ int plan_pos(const int* __restrict__ table, int k) {
    if constexpr (R0 == 0)
        return table[k];
    else
        return dif_pos<R0, R1, R2>(k);
}

// Inverse (DIT) transform with the radix plan fixed at compile time: R0 R1 R2 in the host plan's DIF order
// (R2 = 1 for a two-radix plan), passes run last radix first, as fft_run<true> does at run time.  NB
// transforms, element e of transform b at buf[e * ES + b].  Ends with a barrier.
template <int R0, int R1, int R2, int NB, int ES, int NTHR>
__device__ __forceinline__ void ifft_static(float2* buf, const float2* tw, int tid) {
    constexpr int MM = R0 * R1 * R2;
    if constexpr (R2 > 1) {
        spass<R2, true, true, MM, R2, NB, ES, 1, NTHR>(buf, tw, tid);
        __syncthreads();
    }
    spass<R1, true, true, MM, R1 * R2, NB, ES, 1, NTHR>(buf, tw, tid);
    __syncthreads();
    spass<R0, true, true, MM, MM, NB, ES, 1, NTHR>(buf, tw, tid);
    __syncthreads();
}

}  // namespace dhk
