// Transfer-matrix metrics of a coefficient batch (user guide, AutoAlign section: DIGHOLO_METRIC_IL ... SNRMG,
// digHoloAutoAlignCalcMetrics, digHoloConfigSetAutoAlignBasisMulConjTrans).
//
// The batch is the transfer matrix A [rows = batch][cols = pols x modes] (complex64, as the library writes
// coefficients).  Three kernels, all in FP64 with fixed summation orders:
//   k_gram    Hermitian products A A^H or A^H A (one thread per element of the upper triangle, mirrored);
//   k_jacobi  eigenvalues of the Gram matrix by parallel cyclic Jacobi in one block: round-robin pairings so
//             that n/2 disjoint rotations run at once, each step = rotation parameters, row update, column
//             update, exact zeroing of the rotated pairs; at most kMaxSweeps sweeps (bounded);
//   k_powers  per row of X (= A, or A A^H) the diagonal, row and same-group powers (one warp per row,
//             shuffle tree), then one thread combines rows in order and forms the dB metrics.
#include <cfloat>
#include <cmath>
#include <string>

#include "runtime.hpp"

namespace dhk {
namespace {

constexpr int kJThreads = 1024;
constexpr int kMaxSweeps = 40;

__device__ __forceinline__ double2 ld(const float2* p) { const float2 v = *p; return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 ld(const double2* p) { return *p; }
__device__ __forceinline__ double pw(double2 v) { return v.x * v.x + v.y * v.y; }

// mode group of coefficient index m (modes ordered by group g, which holds g + 1 modes)
__device__ __forceinline__ int group_of(int m) {
    int g = (int)((sqrt(8.0 * m + 1.0) - 1.0) * 0.5);
    while ((g + 1) * (g + 2) / 2 <= m) ++g;
    while (g * (g + 1) / 2 > m) --g;
    return g;
}

// G = A A^H (left = 1: n = rows) or A^H A (left = 0: n = cols)
__global__ void k_gram(const float2* __restrict__ A, int rows, int cols, int left, double2* __restrict__ G, int n) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int i = (int)(idx / n), j = (int)(idx % n);
    if (j < i) return;
    double2 s = make_double2(0.0, 0.0);
    if (left) {
        const float2* a = A + (size_t)i * cols;
        const float2* b = A + (size_t)j * cols;
        for (int k = 0; k < cols; ++k) {   // a_k conj(b_k)
            const double2 x = ld(a + k), y = ld(b + k);
            s.x += x.x * y.x + x.y * y.y;
            s.y += x.y * y.x - x.x * y.y;
        }
    } else {
        for (int k = 0; k < rows; ++k) {   // conj(A_ki) A_kj
            const double2 x = ld(A + (size_t)k * cols + i), y = ld(A + (size_t)k * cols + j);
            s.x += x.x * y.x + x.y * y.y;
            s.y += x.x * y.y - x.y * y.x;
        }
    }
    if (i == j) s.y = 0.0;
    G[(size_t)i * n + j] = s;
    G[(size_t)j * n + i] = make_double2(s.x, -s.y);
}

struct Rot {
    int p, q;
    double cs, sn, a2, b2;
    double2 e;   // exp(-i phi), phi = arg G_pq
};

__device__ void block_sum2(double& a, double& b, double* red) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
        red[2 * w] = a;
        red[2 * w + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            x += red[2 * k];
            y += red[2 * k + 1];
        }
        red[0] = x;
        red[1] = y;
    }
    __syncthreads();
    a = red[0];
    b = red[1];
    __syncthreads();
}

__global__ void __launch_bounds__(kJThreads) k_jacobi(double2* __restrict__ G, int n, double* __restrict__ eig,
                                                      int* __restrict__ sweeps_out) {
    extern __shared__ unsigned char sm[];
    Rot* rot = reinterpret_cast<Rot*>(sm);
    __shared__ double red[2 * (kJThreads / 32)];
    const int np = n + (n & 1);          // padded to even; index n (odd n) is a dummy that never rotates
    const int half = np / 2;
    const int tid = threadIdx.x;
    int sweep = 0;
    for (; sweep < kMaxSweeps; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (long long idx = tid; idx < (long long)n * n; idx += kJThreads) {
            const int i = (int)(idx / n), j = (int)(idx % n);
            const double v = pw(G[idx]);
            if (i == j) dia += v; else off += v;
        }
        block_sum2(off, dia, red);
        if (!(off > 1e-30 * dia)) break;
        for (int step = 0; step < np - 1; ++step) {
            for (int k = tid; k < half; k += kJThreads) {
                const int ja = k, jb = np - 1 - k;
                const int a = ja == 0 ? 0 : 1 + (ja - 1 + step) % (np - 1);
                const int b = 1 + (jb - 1 + step) % (np - 1);
                Rot r;
                r.p = min(a, b);
                r.q = max(a, b);
                r.cs = 1.0;
                r.sn = 0.0;
                r.e = make_double2(1.0, 0.0);
                r.a2 = 0.0;
                r.b2 = 0.0;
                if (r.q < n) {
                    const double app = G[(size_t)r.p * n + r.p].x, aqq = G[(size_t)r.q * n + r.q].x;
                    const double2 c = G[(size_t)r.p * n + r.q];
                    const double h = sqrt(pw(c));
                    r.a2 = app;
                    r.b2 = aqq;
                    if (h > 0.0 && h > 1e-300) {
                        r.e = make_double2(c.x / h, -c.y / h);
                        const double tau = (aqq - app) / (2.0 * h);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        r.cs = 1.0 / sqrt(1.0 + t * t);
                        r.sn = t * r.cs;
                        r.a2 = app - t * h;
                        r.b2 = aqq + t * h;
                    } else {
                        r.q = n;   // nothing to rotate
                    }
                }
                rot[k] = r;
            }
            __syncthreads();
            // rows: (J^H G)_p = cs G_p - sn conj(e) G_q ; (J^H G)_q = sn G_p + cs conj(e) G_q
            for (long long idx = tid; idx < (long long)half * n; idx += kJThreads) {
                const Rot& r = rot[idx / n];
                if (r.q >= n) continue;
                const int c = (int)(idx % n);
                const double2 gp = G[(size_t)r.p * n + c], gq = G[(size_t)r.q * n + c];
                const double2 eq = make_double2(r.e.x * gq.x + r.e.y * gq.y, r.e.x * gq.y - r.e.y * gq.x);   // conj(e) gq
                G[(size_t)r.p * n + c] = make_double2(r.cs * gp.x - r.sn * eq.x, r.cs * gp.y - r.sn * eq.y);
                G[(size_t)r.q * n + c] = make_double2(r.sn * gp.x + r.cs * eq.x, r.sn * gp.y + r.cs * eq.y);
            }
            __syncthreads();
            // columns: (G J)_p = cs G_p - sn e G_q ; (G J)_q = sn G_p + cs e G_q
            for (long long idx = tid; idx < (long long)half * n; idx += kJThreads) {
                const Rot& r = rot[idx / n];
                if (r.q >= n) continue;
                const int row = (int)(idx % n);
                const double2 gp = G[(size_t)row * n + r.p], gq = G[(size_t)row * n + r.q];
                const double2 eq = make_double2(r.e.x * gq.x - r.e.y * gq.y, r.e.x * gq.y + r.e.y * gq.x);   // e gq
                G[(size_t)row * n + r.p] = make_double2(r.cs * gp.x - r.sn * eq.x, r.cs * gp.y - r.sn * eq.y);
                G[(size_t)row * n + r.q] = make_double2(r.sn * gp.x + r.cs * eq.x, r.sn * gp.y + r.cs * eq.y);
            }
            __syncthreads();
            for (int k = tid; k < half; k += kJThreads) {
                const Rot& r = rot[k];
                if (r.q >= n) continue;
                G[(size_t)r.p * n + r.q] = make_double2(0.0, 0.0);
                G[(size_t)r.q * n + r.p] = make_double2(0.0, 0.0);
                G[(size_t)r.p * n + r.p] = make_double2(r.a2, 0.0);
                G[(size_t)r.q * n + r.q] = make_double2(r.b2, 0.0);
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < n; i += kJThreads) eig[i] = G[(size_t)i * n + i].x;
    if (tid == 0) *sweeps_out = sweep;
}

// X [rows][cols] (float2 = A, double2 = A A^H); keys: index -> (pol block, mode group) of a mode index
template <typename E>
__global__ void __launch_bounds__(1024) k_powers(const E* __restrict__ X, int rows, int cols, int modes,
                                                 int grouped, double* __restrict__ rowbuf, const double* __restrict__ eig,
                                                 int n_eig, double* __restrict__ out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < rows; i += nw) {
        const int pi = i / modes, gi = grouped ? group_of(i % modes) : -1;
        double t = 0.0, s = 0.0;
        for (int j = lane; j < cols; j += 32) {
            const double v = pw(ld(X + (size_t)i * cols + j));
            t += v;
            if (grouped && j / modes == pi && group_of(j % modes) == gi) s += v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            t += __shfl_xor_sync(0xffffffffu, t, o);
            s += __shfl_xor_sync(0xffffffffu, s, o);
        }
        if (lane == 0) {
            rowbuf[3 * (size_t)i] = t;
            rowbuf[3 * (size_t)i + 1] = s;
            rowbuf[3 * (size_t)i + 2] = i < cols ? pw(ld(X + (size_t)i * cols + i)) : 0.0;
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    auto db = [inf](double v) { return v > 0.0 ? 10.0 * log10(v) : (v == 0.0 ? -inf : nan("")); };
    auto ratio = [inf](double a, double b) { return b == 0.0 ? inf : a / b; };
    // eigenvalues: below 1e-12 of the largest they count as zero
    double lmax = 0.0;
    for (int k = 0; k < n_eig; ++k) lmax = fmax(lmax, eig[k]);
    double lsum = 0.0, lmin = inf;
    for (int k = 0; k < n_eig; ++k) {
        const double l = eig[k] <= 1e-12 * lmax ? 0.0 : eig[k];
        lsum += l;
        lmin = fmin(lmin, l);
    }
    const int nd = rows < cols ? rows : cols;
    double T = 0.0, S = 0.0, D = 0.0, dmax = -1.0, dmin = inf, smax = -1.0, smin = inf;
    for (int i = 0; i < rows; ++i) {
        const double t = rowbuf[3 * (size_t)i], s = rowbuf[3 * (size_t)i + 1];
        T += t;
        S += s;
        if (i < nd) {
            const double d = rowbuf[3 * (size_t)i + 2];
            D += d;
            dmax = fmax(dmax, d);
            dmin = fmin(dmin, d);
            const double r = ratio(d, t - d);
            smax = fmax(smax, r);
            smin = fmin(smin, r);
        }
    }
    out[0] = db(lsum / n_eig);
    out[1] = db(ratio(lmax, lmin));
    out[2] = db(D);
    out[3] = db(ratio(D, T - D));
    out[4] = db(dmax);
    out[5] = db(dmin);
    out[6] = db(smax);
    out[7] = db(smin);
    out[8] = grouped ? db(ratio(S, T - S)) : -(double)FLT_MAX;
}

}  // namespace
}  // namespace dhk

namespace dh {

static int metrics_impl(Handle* H, const void* d_coefs, int batch, int mct, double* metrics, double* eigenvalues,
                        cudaStream_t st) {
    if (!d_coefs || !metrics) return fail(DH_ERROR_NULLPOINTER, "coefficients or metrics pointer is null");
    if (batch < 1) return fail(DH_ERROR_INVALIDDIMENSION, "batch must be >= 1");
    int rc = ensure_plan(H);
    if (rc) return rc;
    const dhk::Plan& P = H->plan;
    if (P.modes_out == 0) return fail(DH_ERROR_INVALIDDIMENSION, "no coefficients (G = 0)");
    const int cols = P.pols * P.modes_out;
    const int n = std::min(batch, cols);
    if (n > DH_MAX_METRIC_SIZE || (mct && batch > DH_MAX_METRIC_SIZE))
        return fail(DH_ERROR_INVALIDDIMENSION, "transfer matrix larger than DH_MAX_METRIC_SIZE");
    const int xr = batch, xc = mct ? batch : cols;
    const size_t gram = (size_t)n * n * sizeof(double2);
    const size_t xm = mct ? (size_t)batch * batch * sizeof(double2) : 0;
    const size_t rows = (size_t)xr * 3 * sizeof(double);
    const size_t bytes = gram + xm + rows + (size_t)n * sizeof(double) + 16 * sizeof(double) + 256;
    void* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, bytes);
    if (e != cudaSuccess) return fail(DH_ERROR_MEMORYALLOCATION, std::string("metrics scratch: ") + cudaGetErrorString(e));
    unsigned char* b = (unsigned char*)buf;
    double2* G = (double2*)b;
    double2* X = (double2*)(b + gram);
    double* rowbuf = (double*)(b + gram + xm);
    double* eig = rowbuf + (size_t)xr * 3;
    double* out = eig + n;
    int* sweeps = (int*)(out + 9);
    const float2* A = (const float2*)d_coefs;
    const int grouped = (H->geo.basis != DH_BASIS_CUSTOM && P.groups > 0) ? 1 : 0;
    const long long ng = (long long)n * n;
    dhk::k_gram<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(A, batch, cols, batch <= cols ? 1 : 0, G, n);
    if (mct) {
        const long long nx = (long long)batch * batch;
        dhk::k_gram<<<(unsigned)((nx + 255) / 256), 256, 0, st>>>(A, batch, cols, 1, X, batch);
    }
    const int half = (n + (n & 1)) / 2;
    dhk::k_jacobi<<<1, dhk::kJThreads, (size_t)half * sizeof(dhk::Rot), st>>>(G, n, eig, sweeps);
    if (mct)
        dhk::k_powers<double2><<<1, 1024, 0, st>>>(X, xr, xc, P.modes_out, grouped, rowbuf, eig, n, out);
    else
        dhk::k_powers<float2><<<1, 1024, 0, st>>>(A, xr, xc, P.modes_out, grouped, rowbuf, eig, n, out);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(metrics, out, DH_METRIC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && eigenvalues) e = cudaMemcpyAsync(eigenvalues, eig, n * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(buf);
    return e == cudaSuccess ? DH_SUCCESS : cuda_fail(e, "metrics");
}

}  // namespace dh

using namespace dh;

extern "C" int dh_calc_metrics(dh_handle h, const void* d_coefs, int batch, int mul_conj_trans, double* metrics,
                               double* eigenvalues, void* stream) {
    Handle* H = get_handle(h);
    if (!H) return fail(DH_ERROR_INVALIDHANDLE, "invalid handle");
    std::lock_guard<std::mutex> lk(H->mu);
    return metrics_impl(H, d_coefs, batch, mul_conj_trans != 0, metrics, eigenvalues, (cudaStream_t)stream);
}
