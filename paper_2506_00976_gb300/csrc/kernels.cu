// kernels.cu -- device passes of the quantization-based W_p bounds.
//
//   prepare     SumPool of mu and nu (Sec. 2.2) with validation sums
//   cbar        marginally weighted coarse cost C-bar (Sec. 3.2, Alg. 3),
//               reduced over every fine pixel pair of every block pair
//   primal      IPF sweeps of the upscaled plan and its certified cost and
//               TV corrections (Sec. 3.4, Sec. 4, Alg. 4)
//   centre/upsample  bilinear dual upscaling (Sec. 3.5, Alg. 5)
//   ctransform  lazy min-plus c-transform (Sec. 4, eq. lazy c-transform)
//   lbsum       certified dual lower bound (Sec. 3.5, eq. upscaling LB)
//   adjoint     gradient of the lower bound along the simplex
//
// Every kernel takes a list of work items over a table of per-pair
// descriptors, so one launch serves one pair (plain form) or a whole batch of
// pairs with uneven grid sizes (batched form).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

#include <cooperative_groups.h>

namespace qwb {

// --------------------------------------------------------------------------
// Cost tables: tab[dr * N + dc] brackets rho((dr, dc))^p for 0 <= dr, dc < N.
// --------------------------------------------------------------------------
template <typename T>
__global__ void cost_table_kernel(int N, double p, T* lo, T* hi) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * N) return;
    const int dr = idx / N, dc = idx % N;
    if constexpr (sizeof(T) == 4) {
        CostPair<float> c = ground_cost_f32(dr, dc, p);
        lo[idx] = c.lo; hi[idx] = c.hi;
    } else {
        CostPair<double> c = ground_cost_f64(dr, dc, p);
        lo[idx] = c.lo; hi[idx] = c.hi;
    }
}

// 3-D tables: tab[(d1 * N + d2) * N + d3] brackets rho((d1, d2, d3))^p.
template <typename T>
__global__ void cost_table3_kernel(int N, double p, T* lo, T* hi) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * N * N) return;
    const int d1 = idx / (N * N), d2 = (idx / N) % N, d3 = idx % N;
    const double s = (double)d1 * d1 + (double)d2 * d2 + (double)d3 * d3;
    if constexpr (sizeof(T) == 4) {
        CostPair<float> c = ground_cost_sq_f32(s, p);
        lo[idx] = c.lo; hi[idx] = c.hi;
    } else {
        CostPair<double> c = ground_cost_sq_f64(s, p);
        lo[idx] = c.lo; hi[idx] = c.hi;
    }
}

int launch_cost_tables3(int N, double p, bool f64, void* lo, void* hi, cudaStream_t stream) {
    const int n = N * N * N, th = 256, bl = (n + th - 1) / th;
    if (f64) cost_table3_kernel<double><<<bl, th, 0, stream>>>(N, p, (double*)lo, (double*)hi);
    else cost_table3_kernel<float><<<bl, th, 0, stream>>>(N, p, (float*)lo, (float*)hi);
    QWB_LAUNCHED();
    return QWB_OK;
}

// Reflected rows of a lower-bracket table: refl[r * 2N + c + N - 1] = lo[r * N + |c|]
// for |c| < N (the last entry of each row repeats the first one's neighbour
// and is never read).  rows = N (2-D) or N^2 (3-D).
template <typename T>
__global__ void reflect_table_kernel(int N, long rows, const T* lo, T* refl) {
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * 2 * N) return;
    const long r = idx / (2 * N);
    const int cc = (int)(idx - r * 2 * N);
    const int c = min(abs(cc - (N - 1)), N - 1);
    refl[idx] = lo[r * N + c];
}

int launch_reflect_table(int N, int d, bool f64, const void* lo, void* refl, cudaStream_t stream) {
    const long rows = d == 3 ? (long)N * N : N;
    const long n = rows * 2 * N;
    const int th = 256;
    const unsigned bl = (unsigned)((n + th - 1) / th);
    if (f64) reflect_table_kernel<double><<<bl, th, 0, stream>>>(N, rows, (const double*)lo, (double*)refl);
    else reflect_table_kernel<float><<<bl, th, 0, stream>>>(N, rows, (const float*)lo, (float*)refl);
    QWB_LAUNCHED();
    return QWB_OK;
}

int launch_cost_tables(int N, double p, bool f64, void* lo, void* hi, cudaStream_t stream) {
    const int n = N * N, th = 256, bl = (n + th - 1) / th;
    if (f64) cost_table_kernel<double><<<bl, th, 0, stream>>>(N, p, (double*)lo, (double*)hi);
    else cost_table_kernel<float><<<bl, th, 0, stream>>>(N, p, (float*)lo, (float*)hi);
    QWB_LAUNCHED();
    return QWB_OK;
}

// rho(x-bar, x)^p bracket for the TV weights, x-bar = the grid centre
// ((N-1)/2 on every axis); z < 0 for 2-D points.
__device__ __forceinline__ double tv_weight_hi(int r, int c, int N, double p, int z = -1) {
    const double dr = r - 0.5 * (N - 1), dc = c - 0.5 * (N - 1);
    const double dz = z >= 0 ? z - 0.5 * (N - 1) : 0.0;
    const double d2 = dr * dr + dc * dc + dz * dz;        // exact (quarter integers)
    if (p == 2.0) return d2;
    if (p == 1.0) return __dsqrt_ru(d2);
    if (d2 == 0.0) return 0.0;
    return __dmul_ru(pow(d2, 0.5 * p), 1.0 + 0x1p-49);
}

// The same bracket without FP64 arithmetic for p = 1, 2 when N <= 2896:
// 4 |x - x-bar|^2 is an integer below 2^24, exact in FP32; p = 2 returns it
// quartered (exact), p = 1 its square root rounded up, halved (exact).
__device__ __forceinline__ double tv_weight_hi_fast(int r, int c, int N, double p) {
    if ((p == 2.0 || p == 1.0) && N <= 2896) {
        const int dr = 2 * r - (N - 1), dc = 2 * c - (N - 1);
        const float d4 = (float)(dr * dr + dc * dc);
        return widen_f32(p == 2.0 ? 0.25f * d4 : 0.5f * __fsqrt_ru(d4));
    }
    return tv_weight_hi(r, c, N, p);
}

// --------------------------------------------------------------------------
// prepare: SumPool (Sec. 2.2) -- mu~_k = mu(X_k) in FP64, nearest and
// round-down sums, plus validation (finite, non-negative, mass).
// One thread per coarse block; items cover 256 blocks each.
// --------------------------------------------------------------------------
template <typename T>
__global__ void prepare_kernel(const PairDev* __restrict__ pairs, PairOut* __restrict__ outs,
                               const PixItem* __restrict__ items, int n_items) {
    const PixItem I = items[blockIdx.x];
    const PairDev& P = pairs[I.pair];
    const int k = I.start + threadIdx.x;
    double smu = 0.0, snu = 0.0;
    int bad_mu = 0, bad_nu = 0;
    if (k < P.M) {
        const int N = P.N, kap = P.kappa, n = P.n;
        // block coordinates; its kappa^d points in row-major order
        const int k1 = P.d == 3 ? k / (n * n) : k / n;
        const int k2 = P.d == 3 ? (k / n) % n : k % n;
        const int k3 = P.d == 3 ? k % n : 0;
        const int pts = P.d == 3 ? kap * kap * kap : kap * kap;
        double mu_rn = 0.0, mu_rd = 0.0, nu_rn = 0.0, nu_rd = 0.0, mu_ru = 0.0, nu_ru = 0.0;
        double mu_w = 0.0, nu_w = 0.0;
        for (int q = 0; q < pts; ++q) {
            int c1, c2, c3, i;
            if (P.d == 3) {
                c1 = k1 * kap + q / (kap * kap); c2 = k2 * kap + (q / kap) % kap; c3 = k3 * kap + q % kap;
                i = (c1 * N + c2) * N + c3;
            } else {
                c1 = k1 * kap + q / kap; c2 = k2 * kap + q % kap; c3 = -1;
                i = c1 * N + c2;
            }
            const double x = P.mu[i], y = P.nu[i];
            reinterpret_cast<T*>(P.mu_up)[i] = from_double_ru<T>(x);
            reinterpret_cast<T*>(P.nu_up)[i] = from_double_ru<T>(y);
            reinterpret_cast<T*>(P.mu_t)[i] = (T)x;
            reinterpret_cast<T*>(P.nu_t)[i] = (T)y;
            // p = 2 in 2-D: the same (exact) weight without FP64 arithmetic
            const double w = (P.p == 2.0 && P.d == 2 && N <= 2896) ? tv_weight_hi_fast(c1, c2, N, 2.0)
                                                                   : tv_weight_hi(c1, c2, N, P.p, c3);
            mu_w = __fma_ru(w, x, mu_w);
            nu_w = __fma_ru(w, y, nu_w);
            bad_mu |= !(x >= 0.0) || !isfinite(x);
            bad_nu |= !(y >= 0.0) || !isfinite(y);
            mu_rn += x; mu_rd = __dadd_rd(mu_rd, x); mu_ru = __dadd_ru(mu_ru, x);
            nu_rn += y; nu_rd = __dadd_rd(nu_rd, y); nu_ru = __dadd_ru(nu_ru, y);
        }
        P.mu_c[k] = mu_rn; P.mu_c_lo[k] = mu_rd; P.mu_c_hi[k] = mu_ru;
        P.nu_c[k] = nu_rn; P.nu_c_lo[k] = nu_rd; P.nu_c_hi[k] = nu_ru;
        P.mu_w_hi[k] = mu_w; P.nu_w_hi[k] = nu_w;
        // upper bounds of 1 / mu~_k for C-bar (0: zero mass, or too small for FP32)
        P.mu_rinv[k] = mu_rd > 0.0 ? __drcp_ru(mu_rd) : 0.0;
        P.nu_rinv[k] = nu_rd > 0.0 ? __drcp_ru(nu_rd) : 0.0;
        P.mu_rinv32[k] = mu_rd >= 1e-30 ? __frcp_ru(__double2float_rd(mu_rd)) : 0.0f;
        P.nu_rinv32[k] = nu_rd >= 1e-30 ? __frcp_ru(__double2float_rd(nu_rd)) : 0.0f;
        if (sizeof(T) == 4 && P.bsum && P.d == 2) {
            // the block's row and column sums of the rounded-up FP32 masses,
            // rounded up (read back from what this thread wrote above)
            for (int side = 0; side < 2; ++side) {
                const float* up = reinterpret_cast<const float*>(side == 0 ? P.mu_up : P.nu_up) +
                                  (size_t)(k1 * kap) * N + k2 * kap;
                float* dst = P.bsum + ((size_t)side * P.M + k) * 2 * kap;
                for (int a = 0; a < kap; ++a) {
                    float r = 0.0f, c = 0.0f;
                    for (int e = 0; e < kap; ++e) {
                        r = __fadd_ru(r, up[a * N + e]);
                        c = __fadd_ru(c, up[e * N + a]);
                    }
                    dst[a] = r;
                    dst[kap + a] = c;
                }
            }
        }
        smu = mu_rn; snu = nu_rn;
    }
    // block reduction of the masses, one atomic per block
    __shared__ double red[2][32];
    __shared__ int redb[2];
    if (threadIdx.x == 0) { redb[0] = 0; redb[1] = 0; }
    for (int o = 16; o > 0; o >>= 1) {
        smu += __shfl_down_sync(0xffffffffu, smu, o);
        snu += __shfl_down_sync(0xffffffffu, snu, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red[0][warp] = smu; red[1][warp] = snu; }
    __syncthreads();
    if (bad_mu) atomicOr(&redb[0], 1);
    if (bad_nu) atomicOr(&redb[1], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red[0][w]; b += red[1][w]; }
        PairOut& O = outs[P.out_index];
        atomicAdd(&O.mass_mu, a);
        atomicAdd(&O.mass_nu, b);
        if (redb[0]) atomicOr(&O.bad_mu, 1);
        if (redb[1]) atomicOr(&O.bad_nu, 1);
    }
}

int launch_prepare(const PairDev* pairs_d, PairOut* outs_d, const PixItem* items, int n_items,
                   bool f64, cudaStream_t stream) {
    if (n_items <= 0) return QWB_OK;
    if (f64) prepare_kernel<double><<<n_items, 256, 0, stream>>>(pairs_d, outs_d, items, n_items);
    else prepare_kernel<float><<<n_items, 256, 0, stream>>>(pairs_d, outs_d, items, n_items);
    QWB_LAUNCHED();
    return QWB_OK;
}

// --------------------------------------------------------------------------
// cbar: C-bar_kl = [sum_{x in X_k} mu(x) sum_{y in Y_l} nu(y) rho(x,y)^p] /
//                  (mu~_k nu~_l)                       (Sec. 3.2; Alg. 3)
//
// Every fine pixel pair of every block pair contributes one fused multiply-
// add.  Work item = (pair, wrapped block-row diagonal w1, segment): the
// CBAR_S block-row pairs (k1, l1 = (k1 - w1) mod n), k1 = seg*S + s.  Inside a
// block-row pair the n*n block pairs (k2, l2) are walked by wrapped column
// diagonal (slot b: w2 = b / n, k2 = b % n, l2 = (k2 - w2) mod n), so every
// warp gets full, equal work and a thread's block offset (k - l) takes at most
// two values; its (2kappa-1)^2 cost window is held in registers across the S
// block rows.  The staged mu, nu rows and cost-table rows live in shared
// memory; results are staged too and stored as contiguous row segments.
// All products and sums round upward and the division by mu~_k nu~_l is a
// multiplication by upward-rounded reciprocals, so C-bar is bounded from
// above.  A zero-mass block pair gets the unweighted mean of the cost.
// --------------------------------------------------------------------------
constexpr int CBAR_THREADS = 256;

template <typename T>
__device__ __forceinline__ double cbar_special(const PairDev& P, int k, int l, double num,
                                               double mean_up) {
    if (P.mu_c_lo[k] > 0.0 && P.nu_c_lo[l] > 0.0)
        return __dmul_ru(__dmul_ru(num, P.mu_rinv[k]), P.nu_rinv[l]);
    return mean_up;
}

constexpr int CBAR_WPAD = 52;   // (2*4-1)^2 = 49 window entries padded to whole float4s

// Per-thread block-pair slots: slot j of thread t is b = t + j*CBAR_THREADS
// over the n*n pairs (k2, l2), by wrapped column diagonal w2 = b / n.
constexpr int CBAR_MAX_SLOTS = 16;   // n <= 64

template <typename T, int KAP, int MINB>
__global__ void __launch_bounds__(CBAR_THREADS, MINB)
cbar_kernel(const PairDev* __restrict__ pairs, const CbarItem* __restrict__ items, int n_items) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const CbarItem I = items[it];
        const PairDev& P = pairs[I.pair];
        const int N = P.N, n = P.n, M = P.M;
        const int kap = KAP > 0 ? KAP : P.kappa;
        const int W = 2 * kap - 1;
        const int w1 = I.w1;
        double* __restrict__ cbar = P.cbar;
        // shared memory: mu rows [S][kap][N], nu rows [S][kap][N], cost windows,
        // results [S][n][n], reciprocal masses [S][n] twice
        T* mu_s = reinterpret_cast<T*>(smem_raw);
        T* nu_s = mu_s + CBAR_S * kap * N;
        T* win_s = nu_s + CBAR_S * kap * N;
        // KAP > 0: [2][2n-1][CBAR_WPAD] windows, one per (block-row offset, block-column offset)
        // KAP = 0: [2][W][N] cost-table rows for the two block-row offsets
        const int win_len = KAP > 0 ? 2 * (2 * n - 1) * CBAR_WPAD : 2 * W * N;
        T* out_s = win_s + win_len;
        T* rk_s = out_s + CBAR_S * n * n;
        T* rl_s = rk_s + CBAR_S * n;
        const T* tab = reinterpret_cast<const T*>(P.ctab_hi);
        const T* mu_up = reinterpret_cast<const T*>(P.mu_up);   // rounded upward
        const T* nu_up = reinterpret_cast<const T*>(P.nu_up);
        // cost windows of this wrapped block-row diagonal, built once per item
        if constexpr (KAP > 0) {
            constexpr int WK = 2 * KAP - 1;
            for (int vd = threadIdx.x; vd < 2 * (2 * n - 1); vd += blockDim.x) {
                const int v = vd / (2 * n - 1), dd = vd % (2 * n - 1);
                const int D1 = KAP * (v == 0 ? w1 : w1 - n), D2 = KAP * (dd - (n - 1));
                T* dst = win_s + vd * CBAR_WPAD;
#pragma unroll
                for (int d1 = 0; d1 < WK; ++d1) {
                    const int row = abs(D1 + d1 - (KAP - 1));
                    const T* trow = tab + row * N;
#pragma unroll
                    for (int d2 = 0; d2 < WK; ++d2)
                        dst[d1 * WK + d2] = row < N ? trow[abs(D2 + d2 - (KAP - 1))] : T(0);
                }
            }
        } else {
            for (int idx = threadIdx.x; idx < 2 * W * N; idx += blockDim.x) {
                const int v = idx / (W * N), d = (idx / N) % W, c = idx % N;
                const int row = abs(kap * (v == 0 ? w1 : w1 - n) + d - (kap - 1));
                win_s[idx] = row < N ? tab[row * N + c] : T(0);
            }
        }
        // this thread's block-pair slots
        const int n_slots = (n * n + blockDim.x - 1) / blockDim.x;
        int sk2[CBAR_MAX_SLOTS], sl2[CBAR_MAX_SLOTS];
#pragma unroll
        for (int j = 0; j < CBAR_MAX_SLOTS; ++j) {
            const int b = threadIdx.x + j * blockDim.x;
            const int w2 = b / n, k2 = b - w2 * n;
            int l2 = k2 - w2;
            if (l2 < 0) l2 += n;
            sk2[j] = (j < n_slots && b < n * n) ? k2 : -1;
            sl2[j] = l2;
        }
        for (int k1_0 = 0; k1_0 < n; k1_0 += CBAR_S) {
            const int S = min(CBAR_S, n - k1_0);
            __syncthreads();        // previous chunk's results are written out
            // stage rows of mu (block rows k1) and nu (block rows l1 = k1 - w1 mod n)
            const int rowlen = kap * N;
            for (int s = 0; s < S; ++s) {
                const int k1 = k1_0 + s;
                int l1 = k1 - w1;
                if (l1 < 0) l1 += n;
                const T* msrc = mu_up + (size_t)k1 * rowlen;
                const T* nsrc = nu_up + (size_t)l1 * rowlen;
                for (int c = threadIdx.x; c < rowlen; c += blockDim.x) {
                    mu_s[s * rowlen + c] = msrc[c];
                    nu_s[s * rowlen + c] = nsrc[c];
                }
                if (threadIdx.x < n) {
                    if constexpr (sizeof(T) == 4) {
                        rk_s[s * n + threadIdx.x] = P.mu_rinv32[k1 * n + threadIdx.x];
                        rl_s[s * n + threadIdx.x] = P.nu_rinv32[l1 * n + threadIdx.x];
                    } else {
                        rk_s[s * n + threadIdx.x] = P.mu_rinv[k1 * n + threadIdx.x];
                        rl_s[s * n + threadIdx.x] = P.nu_rinv[l1 * n + threadIdx.x];
                    }
                }
            }
            __syncthreads();
            for (int j = 0; j < n_slots; ++j) {
                const int k2 = sk2[j], l2 = sl2[j];
                if (k2 < 0) continue;
                const int D2 = k2 - l2;
                if constexpr (KAP > 0) {
                    constexpr int WK = 2 * KAP - 1;
                    T cw[WK * WK];
                    int cur_v = -1;
                    for (int s = 0; s < S; ++s) {
                        const int k1 = k1_0 + s;
                        const int v = k1 >= w1 ? 0 : 1;          // block-row offset w1 or w1 - n
                        if (v != cur_v) {
                            const T* src = win_s + (v * (2 * n - 1) + D2 + n - 1) * CBAR_WPAD;
                            if constexpr (sizeof(T) == 4 && (WK * WK) % 4 == 1) {
                                float buf[CBAR_WPAD];
#pragma unroll
                                for (int q = 0; q < CBAR_WPAD / 4; ++q)
                                    *reinterpret_cast<float4*>(buf + 4 * q) = reinterpret_cast<const float4*>(src)[q];
#pragma unroll
                                for (int q = 0; q < WK * WK; ++q) cw[q] = buf[q];
                            } else {
#pragma unroll
                                for (int q = 0; q < WK * WK; ++q) cw[q] = src[q];
                            }
                            cur_v = v;
                        }
                        // inner[a] = sum_b nu[b] c(a - b): every nu value feeds KAP^2
                        // independent accumulators (summation order per accumulator
                        // is b1, b2); then acc = sum_a mu[a] inner[a] in order a1, a2
                        T inner[KAP][KAP];
#pragma unroll
                        for (int a1 = 0; a1 < KAP; ++a1)
#pragma unroll
                            for (int a2 = 0; a2 < KAP; ++a2) inner[a1][a2] = T(0);
#pragma unroll
                        for (int b1 = 0; b1 < KAP; ++b1) {
                            T nrow[KAP];
                            const T* np_ = nu_s + (s * KAP + b1) * N + l2 * KAP;
                            if constexpr (KAP == 4 && sizeof(T) == 4) {
                                const float4 v4 = *reinterpret_cast<const float4*>(np_);
                                nrow[0] = v4.x; nrow[1] = v4.y; nrow[2] = v4.z; nrow[3] = v4.w;
                            } else {
#pragma unroll
                                for (int b2 = 0; b2 < KAP; ++b2) nrow[b2] = np_[b2];
                            }
#pragma unroll
                            for (int b2 = 0; b2 < KAP; ++b2)
#pragma unroll
                                for (int a1 = 0; a1 < KAP; ++a1)
#pragma unroll
                                    for (int a2 = 0; a2 < KAP; ++a2)
                                        inner[a1][a2] = fma_ru(nrow[b2], cw[(a1 - b1 + KAP - 1) * WK + a2 - b2 + KAP - 1],
                                                               inner[a1][a2]);
                        }
                        T acc = T(0);
#pragma unroll
                        for (int a1 = 0; a1 < KAP; ++a1) {
                            T mrow[KAP];
                            const T* mp_ = mu_s + (s * KAP + a1) * N + k2 * KAP;
                            if constexpr (KAP == 4 && sizeof(T) == 4) {
                                const float4 v4 = *reinterpret_cast<const float4*>(mp_);
                                mrow[0] = v4.x; mrow[1] = v4.y; mrow[2] = v4.z; mrow[3] = v4.w;
                            } else {
#pragma unroll
                                for (int a2 = 0; a2 < KAP; ++a2) mrow[a2] = mp_[a2];
                            }
#pragma unroll
                            for (int a2 = 0; a2 < KAP; ++a2) acc = fma_ru(mrow[a2], inner[a1][a2], acc);
                        }
                        const T rk = rk_s[s * n + k2], rl = rl_s[s * n + l2];
                        T outv;
                        if (rk > T(0) && rl > T(0)) {
                            outv = mul_ru(mul_ru(acc, rk), rl);
                        } else {
                            int l1 = k1 - w1;
                            if (l1 < 0) l1 += n;
                            const int k = k1 * n + k2, l = l1 * n + l2;
                            double mean = 0.0;
#pragma unroll
                            for (int d1 = 0; d1 < WK; ++d1)
#pragma unroll
                                for (int d2 = 0; d2 < WK; ++d2)
                                    mean = __fma_ru((double)((KAP - abs(d1 - (KAP - 1))) * (KAP - abs(d2 - (KAP - 1)))),
                                                    (double)cw[d1 * WK + d2], mean);
                            mean = __ddiv_ru(mean, (double)(KAP * KAP * KAP * KAP));
                            cbar[(size_t)k * M + l] = cbar_special<T>(P, k, l, (double)acc, mean);
                            outv = sizeof(T) == 4 ? (T)__int_as_float(0x7fc00000) : (T)__longlong_as_double(0x7ff8000000000000LL);
                        }
                        out_s[(s * n + k2) * n + l2] = outv;
                    }
                } else {
                    for (int s = 0; s < S; ++s) {
                        const int k1 = k1_0 + s;
                        const int v = k1 >= w1 ? 0 : 1;
                        const T* cv = win_s + v * W * N;
                        T acc = T(0);
                        double mean = 0.0;
                        for (int a1 = 0; a1 < kap; ++a1)
                            for (int a2 = 0; a2 < kap; ++a2) {
                                const T mv = mu_s[(s * kap + a1) * N + k2 * kap + a2];
                                T inner = T(0);
                                for (int b1 = 0; b1 < kap; ++b1) {
                                    const T* crow = cv + (a1 - b1 + kap - 1) * N;
                                    for (int b2 = 0; b2 < kap; ++b2)
                                        inner = fma_ru(nu_s[(s * kap + b1) * N + l2 * kap + b2],
                                                       crow[abs(kap * D2 + a2 - b2)], inner);
                                }
                                acc = fma_ru(mv, inner, acc);
                            }
                        const T rk = rk_s[s * n + k2], rl = rl_s[s * n + l2];
                        T outv;
                        if (rk > T(0) && rl > T(0)) {
                            outv = mul_ru(mul_ru(acc, rk), rl);
                        } else {
                            int l1 = k1 - w1;
                            if (l1 < 0) l1 += n;
                            const int k = k1 * n + k2, l = l1 * n + l2;
                            for (int a1 = 0; a1 < kap; ++a1)
                                for (int b1 = 0; b1 < kap; ++b1)
                                    for (int a2 = 0; a2 < kap; ++a2)
                                        for (int b2 = 0; b2 < kap; ++b2)
                                            mean = __dadd_ru(mean, (double)cv[(a1 - b1 + kap - 1) * N +
                                                                              abs(kap * D2 + a2 - b2)]);
                            mean = __ddiv_ru(mean, (double)kap * kap * kap * kap);
                            cbar[(size_t)k * M + l] = cbar_special<T>(P, k, l, (double)acc, mean);
                            outv = sizeof(T) == 4 ? (T)__int_as_float(0x7fc00000) : (T)__longlong_as_double(0x7ff8000000000000LL);
                        }
                        out_s[(s * n + k2) * n + l2] = outv;
                    }
                }
            }
            __syncthreads();
            // write the chunk: for each (s, k2) a contiguous row segment of n entries
            for (int rowid = threadIdx.x / n; rowid < S * n; rowid += blockDim.x / n) {
                const int s = rowid / n, k2 = rowid - s * n, l2 = threadIdx.x % n;
                const int k1 = k1_0 + s;
                int l1 = k1 - w1;
                if (l1 < 0) l1 += n;
                const T v = out_s[rowid * n + l2];
                if (v == v)                                          // NaN marks a direct write
                    cbar[(size_t)(k1 * n + k2) * M + l1 * n + l2] = widen_f32(v);
            }
        }
    }
}

// --------------------------------------------------------------------------
// cbar4: the kappa = 4 FP32 C-bar for coarse sides n that are powers of two.
// Same item (one wrapped block-row diagonal w1 of a pair), same sums and
// rounding as cbar_kernel, a different thread mapping: thread slot b covers
// the block pair (k2, l2) = (b / n, b % n) of every staged block row, so the
// threads of a warp hold consecutive target blocks l2 of one source block
// row and write their FP64 results straight to consecutive C-bar entries
// (no staging of outputs, shifts instead of divisions).  Each thread keeps
// the 49 costs of its block offset in registers across the staged rows.
// --------------------------------------------------------------------------
static size_t cbar4_smem(int n, int N, int cs = CBAR_S) {
    return sizeof(float) * ((size_t)2 * cs * 4 * N + (size_t)2 * (2 * n - 1) * CBAR_WPAD + (size_t)2 * cs * n);
}

// CS: block rows staged per chunk (the cost window of a thread's block
// offset is reloaded once per chunk); FIRSTMUL: the first term of each
// accumulator is a round-up product instead of a round-up FMA onto zero (the
// same value: every term is non-negative), so no accumulator is cleared.
template <int MINB, int CS = CBAR_S, bool FIRSTMUL = false>
__global__ void __launch_bounds__(CBAR_THREADS, MINB)
cbar4_kernel(const PairDev* __restrict__ pairs, const CbarItem* __restrict__ items, int n_items) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int KAP = 4, WK = 2 * KAP - 1;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const CbarItem I = items[it];
        const PairDev& P = pairs[I.pair];
        const int N = P.N, n = P.n, M = P.M;
        const int lg = 31 - __clz(n);               // n is a power of two
        const int w1 = I.w1;
        double* __restrict__ cbar = P.cbar;
        float* mu_s = reinterpret_cast<float*>(smem_raw);     // [S][KAP][N]
        float* nu_s = mu_s + CS * KAP * N;                 // [S][KAP][N]
        float* win_s = nu_s + CS * KAP * N;                // [2][2n-1][CBAR_WPAD]
        float* rk_s = win_s + 2 * (2 * n - 1) * CBAR_WPAD;     // [S][n]
        float* rl_s = rk_s + CS * n;                       // [S][n]
        const float* tab = reinterpret_cast<const float*>(P.ctab_hi);
        const float* mu_up = reinterpret_cast<const float*>(P.mu_up);
        const float* nu_up = reinterpret_cast<const float*>(P.nu_up);
        __syncthreads();            // the previous item's readers are done
        for (int vd = threadIdx.x; vd < 2 * (2 * n - 1); vd += blockDim.x) {
            const int v = vd / (2 * n - 1), dd = vd - v * (2 * n - 1);
            const int D1 = KAP * (v == 0 ? w1 : w1 - n), D2 = KAP * (dd - (n - 1));
            float* dst = win_s + vd * CBAR_WPAD;
#pragma unroll
            for (int d1 = 0; d1 < WK; ++d1) {
                const int row = abs(D1 + d1 - (KAP - 1));
                const float* trow = tab + row * N;
#pragma unroll
                for (int d2 = 0; d2 < WK; ++d2)
                    dst[d1 * WK + d2] = row < N ? trow[abs(D2 + d2 - (KAP - 1))] : 0.0f;
            }
        }
        for (int k1_0 = 0; k1_0 < n; k1_0 += CS) {
            const int S = min(CS, n - k1_0);
            __syncthreads();        // windows built / the previous chunk is consumed
            const int rowlen4 = N;  // KAP * N floats = N float4 per block row
            for (int s = 0; s < S; ++s) {
                const int k1 = k1_0 + s;
                int l1 = k1 - w1;
                if (l1 < 0) l1 += n;
                const float4* msrc = reinterpret_cast<const float4*>(mu_up + (size_t)k1 * KAP * N);
                const float4* nsrc = reinterpret_cast<const float4*>(nu_up + (size_t)l1 * KAP * N);
                float4* mdst = reinterpret_cast<float4*>(mu_s + s * KAP * N);
                float4* ndst = reinterpret_cast<float4*>(nu_s + s * KAP * N);
                for (int c = threadIdx.x; c < rowlen4; c += blockDim.x) { mdst[c] = msrc[c]; ndst[c] = nsrc[c]; }
                if (threadIdx.x < n) {
                    rk_s[s * n + threadIdx.x] = P.mu_rinv32[k1 * n + threadIdx.x];
                    rl_s[s * n + threadIdx.x] = P.nu_rinv32[l1 * n + threadIdx.x];
                }
            }
            __syncthreads();
            for (int b = threadIdx.x; b < (n << lg); b += blockDim.x) {
                const int k2 = b >> lg, l2 = b & (n - 1);
                const int D2 = k2 - l2;
                float cw[WK * WK];
                int cur_v = -1;
                for (int s = 0; s < S; ++s) {
                    const int k1 = k1_0 + s;
                    const int v = k1 >= w1 ? 0 : 1;          // block-row offset w1 or w1 - n
                    if (v != cur_v) {
                        const float4* src = reinterpret_cast<const float4*>(
                            win_s + (v * (2 * n - 1) + D2 + n - 1) * CBAR_WPAD);
                        float buf[CBAR_WPAD];
#pragma unroll
                        for (int q = 0; q < CBAR_WPAD / 4; ++q) *reinterpret_cast<float4*>(buf + 4 * q) = src[q];
#pragma unroll
                        for (int q = 0; q < WK * WK; ++q) cw[q] = buf[q];
                        cur_v = v;
                    }
                    // inner[a] = sum_b nu[b] c(a - b) (order b1, b2 per accumulator),
                    // then acc = sum_a mu[a] inner[a] (order a1, a2), all rounded up
                    float inner[KAP][KAP];
                    if constexpr (!FIRSTMUL) {
#pragma unroll
                        for (int a1 = 0; a1 < KAP; ++a1)
#pragma unroll
                            for (int a2 = 0; a2 < KAP; ++a2) inner[a1][a2] = 0.0f;
                    }
#pragma unroll
                    for (int b1 = 0; b1 < KAP; ++b1) {
                        const float4 v4 = *reinterpret_cast<const float4*>(nu_s + (s * KAP + b1) * N + l2 * KAP);
                        const float nrow[KAP] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                        for (int b2 = 0; b2 < KAP; ++b2)
#pragma unroll
                            for (int a1 = 0; a1 < KAP; ++a1)
#pragma unroll
                                for (int a2 = 0; a2 < KAP; ++a2) {
                                    const float c = cw[(a1 - b1 + KAP - 1) * WK + a2 - b2 + KAP - 1];
                                    if (FIRSTMUL && b1 == 0 && b2 == 0) inner[a1][a2] = mul_ru(nrow[b2], c);
                                    else inner[a1][a2] = fma_ru(nrow[b2], c, inner[a1][a2]);
                                }
                    }
                    float acc = 0.0f;
#pragma unroll
                    for (int a1 = 0; a1 < KAP; ++a1) {
                        const float4 v4 = *reinterpret_cast<const float4*>(mu_s + (s * KAP + a1) * N + k2 * KAP);
                        const float mrow[KAP] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                        for (int a2 = 0; a2 < KAP; ++a2) {
                            if (FIRSTMUL && a1 == 0 && a2 == 0) acc = mul_ru(mrow[a2], inner[a1][a2]);
                            else acc = fma_ru(mrow[a2], inner[a1][a2], acc);
                        }
                    }
                    int l1 = k1 - w1;
                    if (l1 < 0) l1 += n;
                    const int k = (k1 << lg) + k2, l = (l1 << lg) + l2;
                    const float rk = rk_s[s * n + k2], rl = rl_s[s * n + l2];
                    double outv;
                    if (rk > 0.0f && rl > 0.0f) {
                        outv = widen_pos_f32(mul_ru(mul_ru(acc, rk), rl));
                    } else {
                        double mean = 0.0;
#pragma unroll
                        for (int d1 = 0; d1 < WK; ++d1)
#pragma unroll
                            for (int d2 = 0; d2 < WK; ++d2)
                                mean = __fma_ru((double)((KAP - abs(d1 - (KAP - 1))) * (KAP - abs(d2 - (KAP - 1)))),
                                                (double)cw[d1 * WK + d2], mean);
                        mean = __ddiv_ru(mean, (double)(KAP * KAP * KAP * KAP));
                        outv = cbar_special<float>(P, k, l, (double)acc, mean);
                    }
                    cbar[(size_t)k * M + l] = outv;
                }
            }
        }
    }
}

// --------------------------------------------------------------------------
// cbar8: the kappa = 8 FP32 C-bar for power-of-two coarse sides n.  Same sums
// and rounding as cbar_kernel (inner[a] = sum_b nu_b c(a - b) over b1, b2,
// then sum_a mu_a inner[a], every FMA rounded up), the thread mapping of
// cbar4 (consecutive target blocks per warp, coalesced FP64 rows).  The
// 15 x 15 cost window of a block offset does not fit in registers, so the
// item stages the 2 x 15 cost-table rows of its two block-row offsets in
// shared memory, reflected (row[c + N - 1] = table[|c|], c in (-N, N)), and a
// thread reads the 15 costs of window row a1 - b1 as four aligned 16-byte
// loads starting at 8 * (k2 - l2) + N - 8; 64 FMAs per window row, in two
// passes of four source rows (32 accumulators).
// --------------------------------------------------------------------------
constexpr int CBAR8_S = 2;   // block rows staged per chunk

static size_t cbar8_smem(int n, int N) {
    return sizeof(float) * ((size_t)2 * 15 * 2 * N + (size_t)2 * CBAR8_S * 8 * N + (size_t)2 * CBAR8_S * n);
}

// A block pair with an empty block (kappa = 8): the unweighted mean of the
// cost over the pair, rounded up, from the staged reflected rows.
__device__ __noinline__ double cbar8_special(const PairDev& P, int k, int l, float acc,
                                             const float* wbase, int RL) {
    constexpr int KAP = 8, WK = 2 * KAP - 1;
    double mean = 0.0;
    for (int d1 = 0; d1 < WK; ++d1)
        for (int d2 = 0; d2 < WK; ++d2)
            mean = __fma_ru((double)((KAP - abs(d1 - (KAP - 1))) * (KAP - abs(d2 - (KAP - 1)))),
                            (double)wbase[d1 * RL + d2], mean);
    mean = __ddiv_ru(mean, (double)(KAP * KAP * KAP * KAP));
    return cbar_special<float>(P, k, l, (double)acc, mean);
}

template <int MINB>
__global__ void __launch_bounds__(CBAR_THREADS, MINB)
cbar8_kernel(const PairDev* __restrict__ pairs, const CbarItem* __restrict__ items, int n_items) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int KAP = 8, WK = 2 * KAP - 1;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const CbarItem I = items[it];
        const PairDev& P = pairs[I.pair];
        const int N = P.N, n = P.n, M = P.M;
        const int lg = 31 - __clz(n);
        const int w1 = I.w1;
        const int RL = 2 * N;                                   // reflected row length (padded)
        double* __restrict__ cbar = P.cbar;
        float* refl_s = reinterpret_cast<float*>(smem_raw);     // [2][15][RL]
        float* mu_s = refl_s + 2 * WK * RL;                     // [S][KAP][N]
        float* nu_s = mu_s + CBAR8_S * KAP * N;                 // [S][KAP][N]
        float* rk_s = nu_s + CBAR8_S * KAP * N;                 // [S][n]
        float* rl_s = rk_s + CBAR8_S * n;                       // [S][n]
        const float* tab = reinterpret_cast<const float*>(P.ctab_hi);
        const float* mu_up = reinterpret_cast<const float*>(P.mu_up);
        const float* nu_up = reinterpret_cast<const float*>(P.nu_up);
        __syncthreads();            // the previous item's readers are done
        for (int idx = threadIdx.x; idx < 2 * WK * RL; idx += blockDim.x) {
            const int vd = idx / RL, c = idx - vd * RL - (N - 1);
            const int v = vd / WK, d1 = vd - v * WK;
            const int row = abs(KAP * (v == 0 ? w1 : w1 - n) + d1 - (KAP - 1));
            refl_s[idx] = (row < N && c < N) ? tab[row * N + abs(c)] : 0.0f;
        }
        for (int k1_0 = 0; k1_0 < n; k1_0 += CBAR8_S) {
            const int S = min(CBAR8_S, n - k1_0);
            __syncthreads();
            for (int s = 0; s < S; ++s) {
                const int k1 = k1_0 + s;
                int l1 = k1 - w1;
                if (l1 < 0) l1 += n;
                const float4* msrc = reinterpret_cast<const float4*>(mu_up + (size_t)k1 * KAP * N);
                const float4* nsrc = reinterpret_cast<const float4*>(nu_up + (size_t)l1 * KAP * N);
                float4* mdst = reinterpret_cast<float4*>(mu_s + s * KAP * N);
                float4* ndst = reinterpret_cast<float4*>(nu_s + s * KAP * N);
                for (int c = threadIdx.x; c < 2 * N; c += blockDim.x) { mdst[c] = msrc[c]; ndst[c] = nsrc[c]; }
                if (threadIdx.x < n) {
                    rk_s[s * n + threadIdx.x] = P.mu_rinv32[k1 * n + threadIdx.x];
                    rl_s[s * n + threadIdx.x] = P.nu_rinv32[l1 * n + threadIdx.x];
                }
            }
            __syncthreads();
            for (int b = threadIdx.x; b < (n << lg); b += blockDim.x) {
                const int k2 = b >> lg, l2 = b & (n - 1);
                const int D2 = k2 - l2;
                for (int s = 0; s < S; ++s) {
                    const int k1 = k1_0 + s;
                    const int v = k1 >= w1 ? 0 : 1;
                    const float* wbase = refl_s + v * WK * RL + KAP * D2 + N - KAP;   // row d1 = 0, col d2 = 0
                    // two passes of four source rows a1 each (32 accumulators)
                    float acc = 0.0f;
#pragma unroll 1
                    for (int ah = 0; ah < KAP; ah += 4) {
                        float inner[4][KAP];
#pragma unroll
                        for (int ar = 0; ar < 4; ++ar)
#pragma unroll
                            for (int a2 = 0; a2 < KAP; ++a2) inner[ar][a2] = 0.0f;
#pragma unroll 1
                        for (int b1 = 0; b1 < KAP; ++b1) {
                            const float4* np4 = reinterpret_cast<const float4*>(nu_s + (s * KAP + b1) * N + l2 * KAP);
                            const float4 n0 = np4[0], n1 = np4[1];
                            const float nrow[KAP] = {n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, n1.z, n1.w};
#pragma unroll
                            for (int ar = 0; ar < 4; ++ar) {
                                const int a1 = ah + ar;
                                const float4* wr = reinterpret_cast<const float4*>(wbase + (a1 - b1 + KAP - 1) * RL);
                                float w[16];
#pragma unroll
                                for (int q = 0; q < 4; ++q) *reinterpret_cast<float4*>(w + 4 * q) = wr[q];
#pragma unroll
                                for (int b2 = 0; b2 < KAP; ++b2)
#pragma unroll
                                    for (int a2 = 0; a2 < KAP; ++a2) {
                                        inner[ar][a2] = fma_ru(nrow[b2], w[a2 - b2 + KAP - 1], inner[ar][a2]);
                                    }
                            }
                        }
#pragma unroll
                        for (int ar = 0; ar < 4; ++ar) {
                            const int a1 = ah + ar;
                            const float4* mp4 = reinterpret_cast<const float4*>(mu_s + (s * KAP + a1) * N + k2 * KAP);
                            const float4 m0 = mp4[0], m1 = mp4[1];
                            const float mrow[KAP] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
                            for (int a2 = 0; a2 < KAP; ++a2) acc = fma_ru(mrow[a2], inner[ar][a2], acc);
                        }
                    }
                    int l1 = k1 - w1;
                    if (l1 < 0) l1 += n;
                    const int k = (k1 << lg) + k2, l = (l1 << lg) + l2;
                    const float rk = rk_s[s * n + k2], rl = rl_s[s * n + l2];
                    cbar[(size_t)k * M + l] = (rk > 0.0f && rl > 0.0f)
                                                  ? widen_pos_f32(mul_ru(mul_ru(acc, rk), rl))
                                                  : cbar8_special(P, k, l, acc, wbase, RL);
                }
            }
        }
    }
}

// --------------------------------------------------------------------------
// cbar3: C-bar on 3-D grids (volumes), the same definition and rounding as
// cbar_kernel: num_kl = sum_{a in X_k} mu_a sum_{b in Y_l} nu_b rho(a, b)^p
// with upward-rounded FMAs (inner sums over b first), then multiplied by
// upward-rounded reciprocals of the block masses.  One CTA per source block
// k stages mu's block; its threads walk the target blocks l.  Costs come from
// the 3-D upper-bracket table tab[(|d1| * N + |d2|) * N + |d3|].
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
cbar3_kernel(const PairDev* __restrict__ pairs, const PixItem* __restrict__ items) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const PixItem I = items[blockIdx.x];
    const PairDev& P = pairs[I.pair];
    const int N = P.N, kap = P.kappa, n = P.n, M = P.M, k = I.start;
    const int pts = kap * kap * kap;
    T* mu_s = reinterpret_cast<T*>(smem_raw);
    const T* mu_up = reinterpret_cast<const T*>(P.mu_up);
    const T* nu_up = reinterpret_cast<const T*>(P.nu_up);
    const T* tab = reinterpret_cast<const T*>(P.ctab_hi);
    const int k1 = k / (n * n), k2 = (k / n) % n, k3 = k % n;
    for (int q = threadIdx.x; q < pts; q += blockDim.x) {
        const int a1 = k1 * kap + q / (kap * kap), a2 = k2 * kap + (q / kap) % kap, a3 = k3 * kap + q % kap;
        mu_s[q] = mu_up[(a1 * N + a2) * N + a3];
    }
    __syncthreads();
    const T rk = sizeof(T) == 4 ? (T)P.mu_rinv32[k] : (T)P.mu_rinv[k];
    for (int l = threadIdx.x; l < M; l += blockDim.x) {
        const int l1 = l / (n * n), l2 = (l / n) % n, l3 = l % n;
        const int D1 = kap * (k1 - l1), D2 = kap * (k2 - l2), D3 = kap * (k3 - l3);
        const int nb = (l1 * kap * N + l2 * kap) * N + l3 * kap;     // first point of Y_l
        T acc = T(0);
        for (int qa = 0; qa < pts; ++qa) {
            const int a1 = qa / (kap * kap), a2 = (qa / kap) % kap, a3 = qa % kap;
            T inner = T(0);
            for (int qb = 0; qb < pts; ++qb) {
                const int b1 = qb / (kap * kap), b2 = (qb / kap) % kap, b3 = qb % kap;
                const int e1 = abs(D1 + a1 - b1), e2 = abs(D2 + a2 - b2), e3 = abs(D3 + a3 - b3);
                inner = fma_ru(nu_up[nb + (b1 * N + b2) * N + b3], tab[(e1 * N + e2) * N + e3], inner);
            }
            acc = fma_ru(mu_s[qa], inner, acc);
        }
        const T rl = sizeof(T) == 4 ? (T)P.nu_rinv32[l] : (T)P.nu_rinv[l];
        double out;
        if (rk > T(0) && rl > T(0)) {
            out = widen_f32(mul_ru(mul_ru(acc, rk), rl));
        } else if (P.mu_c_lo[k] > 0.0 && P.nu_c_lo[l] > 0.0) {
            out = __dmul_ru(__dmul_ru((double)acc, P.mu_rinv[k]), P.nu_rinv[l]);
        } else {                      // a zero-mass block: the unweighted mean cost
            double mean = 0.0;
            for (int qa = 0; qa < pts; ++qa)
                for (int qb = 0; qb < pts; ++qb) {
                    const int e1 = abs(D1 + qa / (kap * kap) - qb / (kap * kap));
                    const int e2 = abs(D2 + (qa / kap) % kap - (qb / kap) % kap);
                    const int e3 = abs(D3 + qa % kap - qb % kap);
                    mean = __dadd_ru(mean, (double)tab[(e1 * N + e2) * N + e3]);
                }
            out = __ddiv_ru(mean, (double)pts * pts);
        }
        P.cbar[(size_t)k * M + l] = out;
    }
}

int launch_cbar3(const PairDev* pairs_d, const PixItem* items, int n_items, bool f64,
                 cudaStream_t stream) {
    if (n_items <= 0) return QWB_OK;
    const size_t smem = (f64 ? 8 : 4) * (size_t)16 * 16 * 16;      // kappa <= 16
    if (f64) cbar3_kernel<double><<<n_items, 256, smem, stream>>>(pairs_d, items);
    else cbar3_kernel<float><<<n_items, 256, smem, stream>>>(pairs_d, items);
    QWB_LAUNCHED();
    return QWB_OK;
}

static size_t cbar_smem(size_t tsz, int kap, int n, int N, bool windows) {
    const size_t win = windows ? (size_t)2 * (2 * n - 1) * CBAR_WPAD : (size_t)2 * (2 * kap - 1) * N;
    return tsz * ((size_t)2 * CBAR_S * kap * N + win + (size_t)CBAR_S * n * n + (size_t)2 * CBAR_S * n);
}

template <typename T>
static int cbar_dispatch(const PairDev* pairs_d, const CbarItem* items, int n_items, int kappa_code,
                         int n_max, int N_max, int variant, cudaStream_t stream) {
    const int kmax = kappa_code > 0 ? kappa_code : -kappa_code;
    const bool windows = kappa_code == 1 || kappa_code == 2 || kappa_code == 4;
    const size_t smem = cbar_smem(sizeof(T), kmax, n_max, N_max, windows);
    auto run = [&](auto kern) -> int {
        if (smem > 227 * 1024) return QWB_ERR_UNSUPPORTED;
        QWB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<n_items, CBAR_THREADS, smem, stream>>>(pairs_d, items, n_items);
        QWB_LAUNCHED();
        return QWB_OK;
    };
    // variant 0: register budget for two CTAs per SM; 1: for three CTAs per SM;
    // 2, 3: the kappa = 4 FP32 kernel with row-direct writes (every coarse side
    // of the launch a power of two), three or two CTAs per SM; 4, 5: the
    // kappa = 8 FP32 kernel (powers of two), two or one CTA per SM; 6, 7, 8:
    // the kappa = 4 kernel with first terms as products, 8 staged rows (6: three
    // CTAs, 7: two CTAs per SM) or 4 (8: three CTAs)
    constexpr int MB = sizeof(T) == 4 ? 3 : 1;
    if constexpr (sizeof(T) == 4) {
        if (kappa_code == 8 && (variant == 4 || variant == 5)) {
            const size_t smem8 = cbar8_smem(n_max, N_max);
            if (smem8 > 227 * 1024) return QWB_ERR_UNSUPPORTED;
            auto kern = variant == 4 ? cbar8_kernel<2> : cbar8_kernel<1>;
            QWB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem8));
            kern<<<n_items, CBAR_THREADS, smem8, stream>>>(pairs_d, items, n_items);
            QWB_LAUNCHED();
            return QWB_OK;
        }
        if (kappa_code == 4 && (variant == 2 || variant == 3 || (variant >= 6 && variant <= 8))) {
            // 6, 7, 8: first terms as products; 8 rows per chunk for 6 and 7
            const int cs = (variant == 6 || variant == 7) ? 8 : CBAR_S;
            const size_t smem4 = cbar4_smem(n_max, N_max, cs);
            if (smem4 > 227 * 1024) return QWB_ERR_UNSUPPORTED;
            auto kern = variant == 2 ? cbar4_kernel<3> : variant == 3 ? cbar4_kernel<2>
                      : variant == 6 ? cbar4_kernel<3, 8, true> : variant == 7 ? cbar4_kernel<2, 8, true>
                                     : cbar4_kernel<3, CBAR_S, true>;
            QWB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem4));
            kern<<<n_items, CBAR_THREADS, smem4, stream>>>(pairs_d, items, n_items);
            QWB_LAUNCHED();
            return QWB_OK;
        }
    }
    switch (kappa_code) {   // positive: every pair of the launch has this kappa
        case 1: return run(cbar_kernel<T, 1, 2>);
        case 2: return run(cbar_kernel<T, 2, 2>);
        case 4: return variant == 1 ? run(cbar_kernel<T, 4, MB>) : run(cbar_kernel<T, 4, 2>);
        default: return run(cbar_kernel<T, 0, 2>);
    }
}

// --------------------------------------------------------------------------
// cbar_sep: C-bar for p = 2 by the separation of the squared distance over
// the two axes.  With x = kappa k + a, y = kappa l + b per axis and
// rho^2 = (x1 - y1)^2 + (x2 - y2)^2, the sum over every fine pixel pair of a
// block pair (Sec. 3.2, the equation that defines C-bar) regroups exactly as
//   sum_{a, b} mu_a nu_b rho^2
//     = sum_{a1} Rmu[a1] sum_{b1} Rnu[b1] (D1 + a1 - b1)^2
//     + sum_{a2} Cmu[a2] sum_{b2} Cnu[b2] (D2 + a2 - b2)^2,
// D = kappa (k - l) per axis, R / C the block's row / column sums.  Every
// term is non-negative and every operation rounds up (from the rounded-up
// FP32 masses and their rounded-up sums), so the entry is an upper bound of
// the real C-bar, as the direct kernels' are; the squares are exact FP32
// integers.  2 kappa^2 + 2 kappa multiply-adds per block pair instead of
// kappa^4 + kappa^2; the first axis's inner sums depend on the target block
// only (the CTA's source block row k1 is fixed), so they are formed once per
// target and reused over the row's n source blocks.  One item per (pair,
// source block row): threads walk the targets l, so every output row is
// written coalesced.  WPRE (coarse sides with n^2 kappa floats in shared
// memory): the second axis's weights Wt[k2][l2][b2] = sum_a2 Cmu[a2]
// (D2 + a2 - b2)^2 depend on the source block and the target's block column
// only, so they are formed once per item and each entry then takes kappa
// multiply-adds per axis (the same rounded-up terms, grouped the other way).
// --------------------------------------------------------------------------
template <int KAP, bool WPRE>
__global__ void __launch_bounds__(256)
cbar_sep_kernel(const PairDev* __restrict__ pairs, const CbarItem* __restrict__ items, int n_items) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int W = 2 * KAP;                               // row sums, then column sums
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const CbarItem I = items[it];
        const PairDev& P = pairs[I.pair];
        const int n = P.n, M = P.M, k1 = I.w1;
        float* ms = reinterpret_cast<float*>(smem_raw);      // [n][W] sums of the row's source blocks
        float* rk_s = ms + n * W;                            // [n] upper bounds of 1 / mu~_k
        __syncthreads();                                     // the previous item's readers are done
        for (int q = threadIdx.x; q < n * W; q += blockDim.x) ms[q] = P.bsum[(size_t)k1 * n * W + q];
        for (int q = threadIdx.x; q < n; q += blockDim.x) rk_s[q] = P.mu_rinv32[k1 * n + q];
        float* wt = rk_s + ((n + 3) & ~3);                   // WPRE: [n][n][KAP], 16-byte aligned
        __syncthreads();
        if constexpr (WPRE) {
            for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
                const int k2 = q / n, l2 = q - k2 * n;
                const float* mk = ms + k2 * W + KAP;           // column sums of source block k2
                const int D2 = KAP * (k2 - l2);
#pragma unroll
                for (int b2 = 0; b2 < KAP; ++b2) {
                    float v = 0.0f;
#pragma unroll
                    for (int a2 = 0; a2 < KAP; ++a2) {
                        const float d = (float)(D2 + a2 - b2);
                        v = fma_ru(mk[a2], d * d, v);
                    }
                    wt[q * KAP + b2] = v;
                }
            }
            __syncthreads();
        }
        const float* nsum = P.bsum + (size_t)M * W;
        for (int l = threadIdx.x; l < M; l += blockDim.x) {
            const int l1 = l / n, l2 = l - l1 * n;
            float Rn[KAP], Cn[KAP];
#pragma unroll
            for (int q = 0; q < KAP; q += 4) {
                const float4 r4 = *reinterpret_cast<const float4*>(nsum + (size_t)l * W + q);
                const float4 c4 = *reinterpret_cast<const float4*>(nsum + (size_t)l * W + KAP + q);
                Rn[q] = r4.x; Rn[q + 1] = r4.y; Rn[q + 2] = r4.z; Rn[q + 3] = r4.w;
                Cn[q] = c4.x; Cn[q + 1] = c4.y; Cn[q + 2] = c4.z; Cn[q + 3] = c4.w;
            }
            const float rl = P.nu_rinv32[l];
            // first axis: V1[a1] = sum_b1 Rnu[b1] (D1 + a1 - b1)^2
            const int D1 = KAP * (k1 - l1);
            float V1[KAP];
#pragma unroll
            for (int a1 = 0; a1 < KAP; ++a1) {
                float v = 0.0f;
#pragma unroll
                for (int b1 = 0; b1 < KAP; ++b1) {
                    const float d = (float)(D1 + a1 - b1);
                    v = fma_ru(Rn[b1], d * d, v);
                }
                V1[a1] = v;
            }
            for (int k2 = 0; k2 < n; ++k2) {
                const float* mk = ms + k2 * W;
                const int D2 = KAP * (k2 - l2);
                float t1 = 0.0f, t2 = 0.0f;
                if constexpr (WPRE) {
                    const float* w = wt + (k2 * n + l2) * KAP;
#pragma unroll
                    for (int a = 0; a < KAP; ++a) {
                        t2 = fma_ru(Cn[a], w[a], t2);
                        t1 = fma_ru(mk[a], V1[a], t1);
                    }
                } else {
                    float sq[2 * KAP - 1];                   // (D2 + e - (KAP - 1))^2, exact
#pragma unroll
                    for (int e = 0; e < 2 * KAP - 1; ++e) {
                        const float d = (float)(D2 + e - (KAP - 1));
                        sq[e] = d * d;
                    }
#pragma unroll
                    for (int a = 0; a < KAP; ++a) {
                        float v = 0.0f;
#pragma unroll
                        for (int b2 = 0; b2 < KAP; ++b2) v = fma_ru(Cn[b2], sq[a - b2 + KAP - 1], v);
                        t2 = fma_ru(mk[KAP + a], v, t2);
                        t1 = fma_ru(mk[a], V1[a], t1);
                    }
                }
                const float acc = __fadd_ru(t1, t2);
                const int k = k1 * n + k2;
                const float rk = rk_s[k2];
                double outv;
                if (rk > 0.0f && rl > 0.0f) {
                    outv = widen_pos_f32(mul_ru(mul_ru(acc, rk), rl));
                } else {
                    // unweighted mean over the block pair: per axis E (D + a - b)^2
                    // = D^2 + (kappa^2 - 1) / 6 for independent uniform a, b
                    const double var = __ddiv_ru((double)(KAP * KAP - 1), 3.0);
                    const double mean = __dadd_ru((double)D1 * D1 + (double)D2 * D2, var);
                    outv = cbar_special<float>(P, k, l, (double)acc, mean);
                }
                P.cbar[(size_t)k * M + l] = outv;
            }
        }
    }
}

int launch_cbar_sep(const PairDev* pairs_d, const CbarItem* items, int n_items, int kappa, int n_max,
                    cudaStream_t stream) {
    if (n_items <= 0) return QWB_OK;
    if (kappa != 4 && kappa != 8) return QWB_ERR_UNSUPPORTED;
    const size_t base = sizeof(float) * ((size_t)n_max * 2 * kappa + ((n_max + 3) & ~3));
    if (base > 48 * 1024) return QWB_ERR_UNSUPPORTED;
    const size_t wpre = base + sizeof(float) * (size_t)n_max * n_max * kappa;
    if (wpre <= 48 * 1024) {
        if (kappa == 4) cbar_sep_kernel<4, true><<<n_items, 256, wpre, stream>>>(pairs_d, items, n_items);
        else cbar_sep_kernel<8, true><<<n_items, 256, wpre, stream>>>(pairs_d, items, n_items);
    } else {
        if (kappa == 4) cbar_sep_kernel<4, false><<<n_items, 256, base, stream>>>(pairs_d, items, n_items);
        else cbar_sep_kernel<8, false><<<n_items, 256, base, stream>>>(pairs_d, items, n_items);
    }
    QWB_LAUNCHED();
    return QWB_OK;
}

int launch_cbar(const PairDev* pairs_d, const CbarItem* items, int n_items, int kappa_code,
                int n_max, int N_max, bool f64, cudaStream_t stream, int variant) {
    if (n_items <= 0) return QWB_OK;
    // kappa_code: the common kappa (1, 2, 4 use unrolled kernels) or -K for a
    // launch whose pairs differ in kappa or use another kappa (largest K)
    if (f64) return cbar_dispatch<double>(pairs_d, items, n_items, kappa_code, n_max, N_max, variant, stream);
    return cbar_dispatch<float>(pairs_d, items, n_items, kappa_code, n_max, N_max, variant, stream);
}

// --------------------------------------------------------------------------
// primal: IPF of pi-hat = pi~ (x) kappa^-4 to (mu, nu) and the certified upper
// bound (Sec. 3.4 IPF paragraph and Theorem; Sec. 4 cost over the support;
// Alg. 4).  One CTA per pair; one thread per coarse block at a time.
//   fine sweeps (type T):  a_i = mu_i / r_k(i),  r = kappa^-4 pi~ B,
//                          b_j = nu_j / s_l(j),  s = kappa^-4 pi~^T A,
//   with A, B the block sums of a, b (b = 1 initially).
//   final FP64 sweep: the same sweep on block scalars (a_i = alpha_k mu_i,
//   b_j = beta_l nu_j, exact for the uniform kernel) defines the certified
//   plan; its marginals, cost and TV corrections are bounded with interval
//   (directed) arithmetic.
// --------------------------------------------------------------------------
constexpr int PRIMAL_THREADS = 256;

__device__ __forceinline__ double block_reduce_ru(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = __dadd_ru(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = __dadd_ru(s, red[w]);
        red[32] = s;
    }
    __syncthreads();
    return red[32];
}
__device__ __forceinline__ double block_reduce_rd(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rd(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = __dadd_rd(s, red[w]);
        red[32] = s;
    }
    __syncthreads();
    return red[32];
}
__device__ __forceinline__ double block_reduce_rn(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        red[32] = s;
    }
    __syncthreads();
    return red[32];
}

// x^(1/p) rounded upward (x >= 0)
__device__ __forceinline__ double root_p_ru(double x, double p) {
    if (x <= 0.0) return 0.0;
    if (p == 1.0) return x;
    if (p == 2.0) return __dsqrt_ru(x);
    return __dmul_ru(pow(x, 1.0 / p), 1.0 + 0x1p-49);
}
__device__ __forceinline__ double root_p_rd(double x, double p) {
    if (x <= 0.0) return 0.0;
    if (p == 1.0) return x;
    if (p == 2.0) return __dsqrt_rd(x);
    return __dmul_rd(pow(x, 1.0 / p), 1.0 - 0x1p-49);
}

// num_kl = sum_{i in X_k} mu_i sum_{j in Y_l} nu_j rho(x_i, y_j)^p with upward
// rounding, accumulated in the same order as the C-bar kernel.
template <typename T, int KAP>
__device__ T block_pair_num(const PairDev& P, int k, int l) {
    const int N = P.N, n = P.n, kap = KAP > 0 ? KAP : P.kappa;
    const int k1 = k / n, k2 = k % n, l1 = l / n, l2 = l % n;
    const T* tab = reinterpret_cast<const T*>(P.ctab_hi);
    const T* mu_up = reinterpret_cast<const T*>(P.mu_up);
    const T* nu_up = reinterpret_cast<const T*>(P.nu_up);
    const int D1 = kap * (k1 - l1), D2 = kap * (k2 - l2);
    T acc = T(0);
    if constexpr (KAP > 0) {
        constexpr int WK = 2 * KAP - 1;
        T cw[WK][WK];
#pragma unroll
        for (int d1 = 0; d1 < WK; ++d1)
#pragma unroll
            for (int d2 = 0; d2 < WK; ++d2)
                cw[d1][d2] = tab[abs(D1 + d1 - (KAP - 1)) * N + abs(D2 + d2 - (KAP - 1))];
        T inner[KAP][KAP];
#pragma unroll
        for (int a1 = 0; a1 < KAP; ++a1)
#pragma unroll
            for (int a2 = 0; a2 < KAP; ++a2) inner[a1][a2] = T(0);
#pragma unroll
        for (int b1 = 0; b1 < KAP; ++b1)
#pragma unroll
            for (int b2 = 0; b2 < KAP; ++b2) {
                const T nv = nu_up[(l1 * KAP + b1) * N + l2 * KAP + b2];
#pragma unroll
                for (int a1 = 0; a1 < KAP; ++a1)
#pragma unroll
                    for (int a2 = 0; a2 < KAP; ++a2)
                        inner[a1][a2] = fma_ru(nv, cw[a1 - b1 + KAP - 1][a2 - b2 + KAP - 1], inner[a1][a2]);
            }
#pragma unroll
        for (int a1 = 0; a1 < KAP; ++a1)
#pragma unroll
            for (int a2 = 0; a2 < KAP; ++a2)
                acc = fma_ru(mu_up[(k1 * KAP + a1) * N + k2 * KAP + a2], inner[a1][a2], acc);
    } else {
        for (int a1 = 0; a1 < kap; ++a1)
            for (int a2 = 0; a2 < kap; ++a2) {
                T inner = T(0);
                for (int b1 = 0; b1 < kap; ++b1)
                    for (int b2 = 0; b2 < kap; ++b2)
                        inner = fma_ru(nu_up[(l1 * kap + b1) * N + l2 * kap + b2],
                                       tab[abs(D1 + a1 - b1) * N + abs(D2 + a2 - b2)], inner);
                acc = fma_ru(mu_up[(k1 * kap + a1) * N + k2 * kap + a2], inner, acc);
            }
    }
    return acc;
}

// The same numerator on 3-D grids (the rounding and order of cbar3_kernel).
template <typename T>
__device__ T block_pair_num3(const PairDev& P, int k, int l) {
    const int N = P.N, n = P.n, kap = P.kappa, pts = kap * kap * kap;
    const T* tab = reinterpret_cast<const T*>(P.ctab_hi);
    const T* mu_up = reinterpret_cast<const T*>(P.mu_up);
    const T* nu_up = reinterpret_cast<const T*>(P.nu_up);
    const int k1 = k / (n * n), k2 = (k / n) % n, k3 = k % n;
    const int l1 = l / (n * n), l2 = (l / n) % n, l3 = l % n;
    const int D1 = kap * (k1 - l1), D2 = kap * (k2 - l2), D3 = kap * (k3 - l3);
    const int mb = (k1 * kap * N + k2 * kap) * N + k3 * kap, nb = (l1 * kap * N + l2 * kap) * N + l3 * kap;
    T acc = T(0);
    for (int qa = 0; qa < pts; ++qa) {
        const int a1 = qa / (kap * kap), a2 = (qa / kap) % kap, a3 = qa % kap;
        T inner = T(0);
        for (int qb = 0; qb < pts; ++qb) {
            const int b1 = qb / (kap * kap), b2 = (qb / kap) % kap, b3 = qb % kap;
            const int e1 = abs(D1 + a1 - b1), e2 = abs(D2 + a2 - b2), e3 = abs(D3 + a3 - b3);
            inner = fma_ru(nu_up[nb + (b1 * N + b2) * N + b3], tab[(e1 * N + e2) * N + e3], inner);
        }
        acc = fma_ru(mu_up[mb + (a1 * N + a2) * N + a3], inner, acc);
    }
    return acc;
}

// Flat index of point t (row-major inside the block) of coarse block k.
__device__ __forceinline__ int block_point(const PairDev& P, int k, int t) {
    const int N = P.N, n = P.n, kap = P.kappa;
    if (P.d == 3) {
        const int k1 = k / (n * n), k2 = (k / n) % n, k3 = k % n;
        return ((k1 * kap + t / (kap * kap)) * N + k2 * kap + (t / kap) % kap) * N + k3 * kap + t % kap;
    }
    return (k / n * kap + t / kap) * N + (k % n) * kap + t % kap;
}

// --------------------------------------------------------------------------
// support_num: the numerators num_kl = sum_{i in X_k, j in Y_l} mu_i nu_j
// rho(x_i, y_j)^p of the plan's support entries (Sec. 4, the cost over
// supp pi-hat; Alg. 4), one thread per entry, with the summation order and
// upward rounding of C-bar.  They depend only on the measures and the
// support, so this pass runs before primal_kernel, which weights them by the
// fitted scalings.  Grid: x over entries (256 per CTA), y over the pairs of
// pair_ids; entries at or past a pair's nnz are skipped, and supp_num holds
// room for every entry of the pair's staged plan.
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
support_num_kernel(const PairDev* __restrict__ pairs, const int* __restrict__ pair_ids) {
    const PairDev& P = pairs[pair_ids[blockIdx.y]];
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P.nnz) return;
    const int M = P.M;
    int lo = 0, hi = M;                      // row of entry e: binary search in rowptr
    while (hi - lo > 1) { const int mid = (lo + hi) >> 1; if (P.rowptr[mid] <= e) lo = mid; else hi = mid; }
    const int k = lo, l = P.colidx[e];
    const T num = P.d == 3 ? block_pair_num3<T>(P, k, l)
                           : (P.kappa == 4 ? block_pair_num<T, 4>(P, k, l) : block_pair_num<T, 0>(P, k, l));
    reinterpret_cast<T*>(P.supp_num)[e] = num;
}

int launch_support_num(const PairDev* pairs_d, const int* pair_ids, int n_pairs, int nnz_max, bool f64,
                       cudaStream_t stream) {
    if (n_pairs <= 0 || nnz_max <= 0) return QWB_OK;
    const dim3 grid((unsigned)((nnz_max + 255) / 256), (unsigned)n_pairs);
    if (f64) support_num_kernel<double><<<grid, 256, 0, stream>>>(pairs_d, pair_ids);
    else support_num_kernel<float><<<grid, 256, 0, stream>>>(pairs_d, pair_ids);
    QWB_LAUNCHED();
    return QWB_OK;
}

template <typename T>
__global__ void __launch_bounds__(PRIMAL_THREADS, 2)
primal_kernel(const PairDev* __restrict__ pairs, PairOut* __restrict__ outs,
              const int* __restrict__ pair_ids, int csr_cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[33];
    const PairDev& P = pairs[pair_ids[blockIdx.x]];
    const int N = P.N, kap = P.kappa, n = P.n, M = P.M;
    double* Bd = reinterpret_cast<double*>(smem_raw);    // FP64 phase: block sums of b
    double* Ad = Bd + M;                                  //             block sums of a
    double* alpha = Ad + M;                               //             a_i = alpha_k mu_i
    double* beta = alpha + M;                             //             b_j = beta_l nu_j
    T* Bt = reinterpret_cast<T*>(beta + M);               // fine phase block sums
    T* At = Bt + M;
    T* a = reinterpret_cast<T*>(P.a);
    T* b = reinterpret_cast<T*>(P.b);
    const int kpts = P.d == 3 ? kap * kap * kap : kap * kap;     // points per block, kappa^d
    const T kinvK = T(1) / (T)((double)kpts * kpts);             // the kernel value kappa^-2d
    const T kk = (T)kpts;

    // the coarse plan's CSR and CSC (indices and pass-type values), staged in
    // shared memory when they fit: every sweep walks them twice
    const int* rp = P.rowptr;
    const int* ci = P.colidx;
    const int* cp = P.colptr;
    const int* ri = P.rowidx;
    const T* vt = reinterpret_cast<const T*>(P.val_t);
    const T* vct = reinterpret_cast<const T*>(P.valc_t);
    if (P.nnz <= csr_cap) {
        T* v_s = At + M;
        T* vc_s = v_s + csr_cap;
        int* rp_s = reinterpret_cast<int*>(vc_s + csr_cap);
        int* cp_s = rp_s + (M + 1);
        int* ci_s = cp_s + (M + 1);
        int* ri_s = ci_s + csr_cap;
        for (int k = threadIdx.x; k <= M; k += blockDim.x) { rp_s[k] = rp[k]; cp_s[k] = cp[k]; }
        for (int e = threadIdx.x; e < P.nnz; e += blockDim.x) {
            ci_s[e] = ci[e]; ri_s[e] = ri[e]; v_s[e] = vt[e]; vc_s[e] = vct[e];
        }
        rp = rp_s; ci = ci_s; cp = cp_s; ri = ri_s; vt = v_s; vct = vc_s;
    }

    // ---- fine sweeps ------------------------------------------------------
    const T* mu_t = reinterpret_cast<const T*>(P.mu_t);    // written by the SumPool pass
    const T* nu_t = reinterpret_cast<const T*>(P.nu_t);
    for (int l = threadIdx.x; l < M; l += blockDim.x) Bt[l] = kk;    // b = 1
    __syncthreads();
    const bool vec4 = (sizeof(T) == 4) && (kap == 4) && P.d == 2;  // block rows are one float4
    const int fine_sweeps = P.fine_ext ? 0 : P.sweeps;     // else done by ipf_fine_kernel
    for (int sweep = 0; sweep < fine_sweeps; ++sweep) {
        for (int half = 0; half < 2; ++half) {
            // half 0: a = mu / (pi-hat b), A = block sums of a
            // half 1: b = nu / (pi-hat^T a), B = block sums of b
            const int* ptr = half == 0 ? rp : cp;
            const int* idx = half == 0 ? ci : ri;
            const T* val = half == 0 ? vt : vct;
            const T* src = half == 0 ? mu_t : nu_t;
            T* dst = half == 0 ? a : b;
            const T* other = half == 0 ? Bt : At;
            T* mine = half == 0 ? At : Bt;
            if (vec4) {
                // up to four blocks per thread at a time: all their fine rows
                // are requested before the first coarse matvec, so a half
                // sweep waits for one memory round trip
                const float* srcf = reinterpret_cast<const float*>(src);
                float* dstf = reinterpret_cast<float*>(dst);
                for (int kb = threadIdx.x; kb < M; kb += 4 * blockDim.x) {
                    float4 x[4][4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int k = kb + q * blockDim.x;
                        if (k < M) {
                            const int k1 = k / n, k2 = k - (k / n) * n;
#pragma unroll
                            for (int t1 = 0; t1 < 4; ++t1)
                                x[q][t1] = *reinterpret_cast<const float4*>(srcf + (k1 * 4 + t1) * N + k2 * 4);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int k = kb + q * blockDim.x;
                        if (k < M) {
                            T r = T(0);
                            for (int e = ptr[k]; e < ptr[k + 1]; ++e) r += val[e] * other[idx[e]];
                            r *= kinvK;
                            const float inv = r > T(0) ? (float)(T(1) / r) : 0.0f;
                            const int k1 = k / n, k2 = k - (k / n) * n;
                            T s = T(0);
#pragma unroll
                            for (int t1 = 0; t1 < 4; ++t1) {
                                float4 v = x[q][t1];
                                v.x *= inv; v.y *= inv; v.z *= inv; v.w *= inv;
                                *reinterpret_cast<float4*>(dstf + (k1 * 4 + t1) * N + k2 * 4) = v;
                                s += (T)((v.x + v.y) + (v.z + v.w));
                            }
                            mine[k] = s;
                        }
                    }
                }
            } else {
                for (int k = threadIdx.x; k < M; k += blockDim.x) {
                    T r = T(0);
                    for (int e = ptr[k]; e < ptr[k + 1]; ++e) r += val[e] * other[idx[e]];
                    r *= kinvK;
                    const T inv = r > T(0) ? T(1) / r : T(0);
                    T s = T(0);
                    for (int t = 0; t < kpts; ++t) {
                        const int i = block_point(P, k, t);
                        const T v = src[i] * inv;
                        dst[i] = v;
                        s += v;
                    }
                    mine[k] = s;
                }
            }
            __syncthreads();
        }
    }

    // ---- FP64 sweeps on block scalars until the marginals are exact --------
    // With the uniform kernel a_i / mu_i and b_j / nu_j stay constant on each
    // block, so a sweep acts on alpha_k, beta_l exactly.  The FP64 sweeps
    // start, as Alg. 4 does, from b = 1 (block sums kappa^2): from there the
    // fixed point is reached after one sweep, whereas from the rounded FP32
    // state IPF on the tree-shaped support of pi~ barely contracts.  They stop
    // once the FP64 residual is at rounding level (at most four sweeps).
    const double k4 = (double)kpts * kpts;                       // kappa^2d
    const double kinv4_rn = 1.0 / k4, kinv4_lo = __drcp_rd(k4), kinv4_hi = __drcp_ru(k4);
    for (int l = threadIdx.x; l < M; l += blockDim.x) Bd[l] = (double)kpts;
    __syncthreads();
    int fp64_sweeps = 0;
    for (;;) {
        for (int k = threadIdx.x; k < M; k += blockDim.x) {        // a = mu / (pi-hat b)
            double r = 0.0;
            for (int e = rp[k]; e < rp[k + 1]; ++e) r += P.val[e] * Bd[ci[e]];
            r *= kinv4_rn;
            alpha[k] = r > 0.0 ? 1.0 / r : 0.0;
            Ad[k] = alpha[k] * P.mu_c[k];
        }
        __syncthreads();
        for (int l = threadIdx.x; l < M; l += blockDim.x) {        // b = nu / (pi-hat^T a)
            double s = 0.0;
            for (int e = cp[l]; e < cp[l + 1]; ++e) s += P.valc[e] * Ad[ri[e]];
            s *= kinv4_rn;
            beta[l] = s > 0.0 ? 1.0 / s : 0.0;
        }
        __syncthreads();
        ++fp64_sweeps;
        double res = 0.0;                                         // ||mu-hat - mu||_1
        for (int k = threadIdx.x; k < M; k += blockDim.x) {
            double s = 0.0;
            for (int e = rp[k]; e < rp[k + 1]; ++e) s += P.val[e] * beta[ci[e]] * P.nu_c[ci[e]];
            res += fabs(alpha[k] * kinv4_rn * s - 1.0) * P.mu_c[k];
        }
        res = block_reduce_rn(res, red);
        if (res <= 4e-15 || fp64_sweeps >= 4) break;
        for (int l = threadIdx.x; l < M; l += blockDim.x) Bd[l] = beta[l] * P.nu_c[l];
        __syncthreads();
    }
    // the certified plan is pi-hat_xi(i,j) = alpha_k mu_i kappa^-4 pi~_kl beta_l nu_j
    if (P.a_out)
        for (int k = threadIdx.x; k < M; k += blockDim.x)
            for (int t = 0; t < kpts; ++t) {
                const int i = block_point(P, k, t);
                P.a_out[i] = alpha[k] * P.mu[i];
            }
    if (P.b_out)
        for (int l = threadIdx.x; l < M; l += blockDim.x)
            for (int t = 0; t < kpts; ++t) {
                const int j = block_point(P, l, t);
                P.b_out[j] = beta[l] * P.nu[j];
            }

    // ---- certified marginals and TV sums ---------------------------------
    // rho_k = alpha_k kappa^-4 sum_l pi~_kl beta_l nu~_l ;  mu-hat = rho_k mu
    double tv_mu = 0.0, res_mu = 0.0;
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
        const double m_hi = P.mu_c_hi[k], w_hi = P.mu_w_hi[k];
        double s_lo = 0.0, s_hi = 0.0;
        for (int e = rp[k]; e < rp[k + 1]; ++e) {
            const int l = ci[e];
            s_lo = __fma_rd(__dmul_rd(P.val[e], beta[l]), P.nu_c_lo[l], s_lo);
            s_hi = __fma_ru(__dmul_ru(P.val[e], beta[l]), P.nu_c_hi[l], s_hi);
        }
        const double rho_lo = __dmul_rd(__dmul_rd(alpha[k], kinv4_lo), s_lo);
        const double rho_hi = __dmul_ru(__dmul_ru(alpha[k], kinv4_hi), s_hi);
        double dev = fmax(0.0, fmax(__dsub_ru(rho_hi, 1.0), __dsub_ru(1.0, rho_lo)));
        if (m_hi == 0.0) dev = 0.0;    // empty block: mu-hat = mu = 0 there
        tv_mu = __fma_ru(dev, w_hi, tv_mu);
        res_mu += fabs(0.5 * (rho_lo + rho_hi) - 1.0) * P.mu_c[k];
    }
    double tv_nu = 0.0, res_nu = 0.0;
    for (int l = threadIdx.x; l < M; l += blockDim.x) {
        const double m_hi = P.nu_c_hi[l], w_hi = P.nu_w_hi[l];
        double s_lo = 0.0, s_hi = 0.0;
        for (int e = cp[l]; e < cp[l + 1]; ++e) {
            const int k = ri[e];
            s_lo = __fma_rd(__dmul_rd(P.valc[e], alpha[k]), P.mu_c_lo[k], s_lo);
            s_hi = __fma_ru(__dmul_ru(P.valc[e], alpha[k]), P.mu_c_hi[k], s_hi);
        }
        const double sg_lo = __dmul_rd(__dmul_rd(beta[l], kinv4_lo), s_lo);
        const double sg_hi = __dmul_ru(__dmul_ru(beta[l], kinv4_hi), s_hi);
        double dev = fmax(0.0, fmax(__dsub_ru(sg_hi, 1.0), __dsub_ru(1.0, sg_lo)));
        if (m_hi == 0.0) dev = 0.0;
        tv_nu = __fma_ru(dev, w_hi, tv_nu);
        res_nu += fabs(0.5 * (sg_lo + sg_hi) - 1.0) * P.nu_c[l];
    }

    // ---- certified cost of the fitted plan over its support -----------------
    // W-hat^p = sum_{(k,l) in supp pi~} kappa^-4 pi~_kl alpha_k beta_l num_kl,
    // num_kl = sum_{i in X_k, j in Y_l} mu_i nu_j rho(x_i, y_j)^p (rounded up)
    double cost = 0.0;
    for (int e = threadIdx.x; e < P.nnz; e += blockDim.x) {
        // row of entry e: binary search in rowptr
        int lo = 0, hi = M;
        while (hi - lo > 1) { const int mid = (lo + hi) >> 1; if (rp[mid] <= e) lo = mid; else hi = mid; }
        const int k = lo, l = ci[e];
        const T num = reinterpret_cast<const T*>(P.supp_num)[e];    // support_num_kernel
        const double term = __dmul_ru(__dmul_ru(__dmul_ru(__dmul_ru(P.val[e], kinv4_hi), alpha[k]), beta[l]),
                                      (double)num);
        cost = __dadd_ru(cost, term);
    }
    const double cost_sum = block_reduce_ru(cost, red);
    const double tvm = block_reduce_ru(tv_mu, red);
    const double tvn = block_reduce_ru(tv_nu, red);
    const double rm = block_reduce_rn(res_mu, red);
    const double rn = block_reduce_rn(res_nu, red);
    if (threadIdx.x == 0) {
        const double p = P.p;
        // Delta = 2^(1-1/p) <w, |.|>^(1/p) = (2^(p-1) <w, |.|>)^(1/p)
        const double scale = (p == 1.0) ? 1.0 : (p == 2.0 ? 2.0 : __dmul_ru(pow(2.0, p - 1.0), 1.0 + 0x1p-49));
        const double dmu = root_p_ru(__dmul_ru(scale, tvm), p);
        const double dnu = root_p_ru(__dmul_ru(scale, tvn), p);
        const double w_hat = root_p_ru(cost_sum, p);
        PairOut& O = outs[P.out_index];
        O.w_hat_p = cost_sum;
        O.delta_mu = dmu;
        O.delta_nu = dnu;
        O.ub_primal = __dadd_ru(__dadd_ru(w_hat, dmu), dnu);
        O.ipf_residual = rm + rn;
        O.sweeps_done = P.sweeps + fp64_sweeps;
    }
}

int launch_primal(const PairDev* pairs_d, PairOut* outs_d, const int* pair_ids, int n_pairs,
                  int M_max, int nnz_max, bool f64, cudaStream_t stream) {
    if (n_pairs <= 0) return QWB_OK;
    const size_t tsz = f64 ? 8 : 4;
    const size_t base = 4 * sizeof(double) * (size_t)M_max + 2 * tsz * (size_t)M_max;
    if (base > 220 * 1024) return QWB_ERR_UNSUPPORTED;
    // stage the plan in shared memory when it fits next to two CTAs per SM
    // (network simplex plans have at most 2M - 1 entries)
    const int cap = std::max(nnz_max, 2 * M_max);
    const size_t csr = 2 * (tsz + sizeof(int)) * (size_t)cap + 2 * sizeof(int) * (size_t)(M_max + 1);
    const bool staged = base + csr <= 110 * 1024;
    const size_t smem = staged ? base + csr : base;
    const int csr_cap = staged ? cap : -1;
    if (f64) {
        QWB_CUDA(cudaFuncSetAttribute(primal_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        primal_kernel<double><<<n_pairs, PRIMAL_THREADS, smem, stream>>>(pairs_d, outs_d, pair_ids, csr_cap);
    } else {
        QWB_CUDA(cudaFuncSetAttribute(primal_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        primal_kernel<float><<<n_pairs, PRIMAL_THREADS, smem, stream>>>(pairs_d, outs_d, pair_ids, csr_cap);
    }
    QWB_LAUNCHED();
    return QWB_OK;
}

// --------------------------------------------------------------------------
// primalk: the primal upscaling upper bound with a general normalized
// positive kernel K (Sec. 3.4, eq. coupling tensor upscale; Alg. 4), d = 2,
// kappa <= 8.  pi-hat_ij = pi~_{k(i) l(j)} K[u(i), v(j)], with u, v the
// row-major offsets of i, j in their blocks.  One CTA per pair.  The
// scalings a, b live block-major ([block][offset], position t = k kk + u with
// kk = kappa^2), so a block's values are one contiguous row.
//   fine sweeps (type T): a = mu / (pi-hat b), b = nu / (pi-hat^T a) from
//     b = 1.  With KB[l, u] = sum_w K[u, w] b[l, w] (and KA[k, v] = sum_w
//     K[w, v] a[k, w]) the a half is r[k, u] = sum_l pi~_kl KB[l, u],
//     a = mu / r, the b half the same with KA and the plan's columns.
//   certified evaluation (FP64 bounds, directed rounding) of the plan
//     diag(a) pi-hat' diag(b) with the final a, b as they are, pi-hat' built
//     with the kernel K' in the pass type (the FP32-rounded K for MIXED, K
//     itself for F64; any positive kernel gives a valid bound): bounds of
//     its marginals and of its total mass s, its cost over the support
//     rounded up and divided by s rounded down (the plan over s couples the
//     probability measures mu-hat / s and nu-hat / s), and the weighted-TV
//     corrections between those and mu, nu.
// FP32 with kappa 2, 4 or 8 (kk = 4, 16, 64) runs the fused sweep: a thread
// owns the four consecutive offsets 4g..4g+3 of one block, the q4 = kk / 4
// lanes of a block hold its whole row, so after r and the new scaling the
// next half's product (KA from a, KB from b) follows from warp shuffles of
// that row -- one barrier per half, KA and KB double-buffered (shared memory
// when they fit).  Other cases run two steps per half (product, barrier,
// gather).
// --------------------------------------------------------------------------
constexpr int PRIMALK_THREADS_F32 = 1024;
constexpr int PRIMALK_THREADS_F64 = 512;

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__device__ __forceinline__ int blk_pixel(int k, int u, int n, int kap, int N) {
    return ((k / n) * kap + u / kap) * N + (k % n) * kap + u % kap;
}

// s / r for the FP32 sweeps (0 where r <= 0): the approximate reciprocal
// refined by one Newton step, within a few ulp (the sweeps are not part of
// the certificate, which takes the final scalings as they are); tiny r takes
// and huge r take the IEEE division, so no denormal is flushed.
__device__ __forceinline__ float ipf_div(float s, float r) {
    if (!(r > 0x1p-100f && r < 0x1p100f)) return r > 0.f ? s / r : 0.f;
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r));
    y = fmaf(y, fmaf(-r, y, 1.0f), y);
    return s * y;
}

// one fused-sweep update: r = sum_e pi~_e KIN[idx_e, 4g..4g+3], x = src / r
__device__ __forceinline__ float4 primalk_update(int k, int g, int q4, const int* ptr, const int* idx,
                                                 const float* val, const float4* kin4, float4 sv) {
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = ptr[k]; e < ptr[k + 1]; ++e) {
        const float v = val[e];
        const float4 kv = kin4[idx[e] * q4 + g];
        r.x = fmaf(v, kv.x, r.x);
        r.y = fmaf(v, kv.y, r.y);
        r.z = fmaf(v, kv.z, r.z);
        r.w = fmaf(v, kv.w, r.w);
    }
    return make_float4(ipf_div(sv.x, r.x), ipf_div(sv.y, r.y), ipf_div(sv.z, r.z), ipf_div(sv.w, r.w));
}

// s += sum_j K'[4 w4 + j][4g..4g+3] x_(4 w4 + j), the four x taken from lane `src`
__device__ __forceinline__ void primalk_row_fma(float4& s, const float4 xv, int src, const float4 k0,
                                                const float4 k1, const float4 k2, const float4 k3) {
    const float x0 = __shfl_sync(0xffffffffu, xv.x, src);
    const float x1 = __shfl_sync(0xffffffffu, xv.y, src);
    const float x2 = __shfl_sync(0xffffffffu, xv.z, src);
    const float x3 = __shfl_sync(0xffffffffu, xv.w, src);
    s.x = fmaf(k3.x, x3, fmaf(k2.x, x2, fmaf(k1.x, x1, fmaf(k0.x, x0, s.x))));
    s.y = fmaf(k3.y, x3, fmaf(k2.y, x2, fmaf(k1.y, x1, fmaf(k0.y, x0, s.y))));
    s.z = fmaf(k3.z, x3, fmaf(k2.z, x2, fmaf(k1.z, x1, fmaf(k0.z, x0, s.z))));
    s.w = fmaf(k3.w, x3, fmaf(k2.w, x2, fmaf(k1.w, x1, fmaf(k0.w, x0, s.w))));
}

// err-free product and sum in FP32 (Dekker / Knuth via FMA)
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& t) {
    s = a + b;
    const float bp = s - a;
    t = (a - (s - bp)) + (b - bp);
}

template <typename T, int KK>
__global__ void __launch_bounds__(sizeof(T) == 4 ? PRIMALK_THREADS_F32 : PRIMALK_THREADS_F64, 1)
primalk_kernel(const PairDev* __restrict__ pairs, PairOut* __restrict__ outs,
               const int* __restrict__ pair_ids, int csr_cap, int kk_max, int kb_cap, int sweeps_only) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[33];
    const PairDev& P = pairs[pair_ids[blockIdx.x]];
    const int N = P.N, kap = P.kappa, n = P.n, m = P.m, M = P.M;
    const int kk = KK ? KK : kap * kap;                       // kk_max: the launch's smem layout
    const int q4 = KK ? KK / 4 : kk >> 2;                      // float4s per block row
    const bool fused = sizeof(T) == 4 && (kk == 4 || kk == 16 || kk == 64);
    // shared memory: [K (T) | K^T (T) | KB, KA (kb_cap each, when > 0) | staged plan]
    const size_t kq = (size_t)kk_max * kk_max;
    const size_t o_kst = align16(sizeof(T) * kq), o_kb = 2 * align16(sizeof(T) * kq),
                 o_csr = o_kb + 2 * align16(sizeof(T) * (size_t)kb_cap);
    T* Ks = reinterpret_cast<T*>(smem_raw);                   // K'[u][w] (row w: K'[w][.])
    T* KsT = reinterpret_cast<T*>(smem_raw + o_kst);          // row w: K'[.][w]
    for (int t = threadIdx.x; t < kk * kk; t += blockDim.x) {
        const int u = t / kk, w = t - (t / kk) * kk;
        const T kt = reinterpret_cast<const T*>(P.upK_t)[t];
        Ks[t] = kt;
        KsT[w * kk + u] = kt;
    }
    // the coarse plan's CSR and CSC, staged in shared memory when they fit
    const int* rp = P.rowptr;
    const int* ci = P.colidx;
    const int* cp = P.colptr;
    const int* ri = P.rowidx;
    const T* vt = reinterpret_cast<const T*>(P.val_t);
    const T* vct = reinterpret_cast<const T*>(P.valc_t);
    const double* v64 = P.val;
    if (P.nnz <= csr_cap) {
        // [v64 (8 cap) | v, vc (T, cap each) | rowptr, colptr (M_max + 1 each) | colidx, rowidx (cap each)]
        double* v64_s = reinterpret_cast<double*>(smem_raw + o_csr);
        T* v_s = reinterpret_cast<T*>(v64_s + csr_cap);
        T* vc_s = v_s + csr_cap;
        int* rp_s = reinterpret_cast<int*>(vc_s + csr_cap);
        int* cp_s = rp_s + (M + 1);
        int* ci_s = cp_s + (M + 1);
        int* ri_s = ci_s + csr_cap;
        for (int q = threadIdx.x; q <= M; q += blockDim.x) { rp_s[q] = rp[q]; cp_s[q] = cp[q]; }
        for (int e = threadIdx.x; e < P.nnz; e += blockDim.x) {
            ci_s[e] = ci[e]; ri_s[e] = ri[e]; v_s[e] = vt[e]; vc_s[e] = vct[e]; v64_s[e] = v64[e];
        }
        rp = rp_s; ci = ci_s; cp = cp_s; ri = ri_s; vt = v_s; vct = vc_s; v64 = v64_s;
    }
    T* a = reinterpret_cast<T*>(P.a);
    T* b = reinterpret_cast<T*>(P.b);
    // KB (read by the a half) and KA (read by the b half)
    T* kbB = m <= kb_cap ? reinterpret_cast<T*>(smem_raw + o_kb) : reinterpret_cast<T*>(P.kb_t);
    T* kbA = m <= kb_cap ? reinterpret_cast<T*>(smem_raw + o_kb + align16(sizeof(T) * (size_t)kb_cap))
                         : reinterpret_cast<T*>(P.kb_t) + m;
    T* mu_b = reinterpret_cast<T*>(P.kscratch);               // block-major copies of mu, nu (sweeps only)
    T* nu_b = mu_b + m;
    const T* mu_t = reinterpret_cast<const T*>(P.mu_t);
    const T* nu_t = reinterpret_cast<const T*>(P.nu_t);
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        const int i = blk_pixel(t / kk, t - (t / kk) * kk, n, kap, N);
        mu_b[t] = mu_t[i];
        nu_b[t] = nu_t[i];
        b[t] = T(1);
    }
    __syncthreads();
    // ---- fine sweeps ------------------------------------------------------
    if (fused) {
        const float4* Ks4 = reinterpret_cast<const float4*>(Ks);
        const float4* KsT4 = reinterpret_cast<const float4*>(KsT);
        const int n_items = m >> 2;
        const int n_iter = (n_items + blockDim.x - 1) / blockDim.x;   // the same for every thread
        const int lane = threadIdx.x & 31;
        // b = 1: KB[l, u] = sum_w K'[u][w]
        for (int it = threadIdx.x; it < n_items; it += blockDim.x) {
            const int g = it % q4;
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int w = 0; w < kk; ++w) {
                const float4 kv = KsT4[w * q4 + g];
                s.x += kv.x; s.y += kv.y; s.z += kv.z; s.w += kv.w;
            }
            reinterpret_cast<float4*>(kbB)[it] = s;
        }
        __syncthreads();
        for (int sweep = 0; sweep < P.sweeps; ++sweep) {
            for (int half = 0; half < 2; ++half) {
                const int* ptr = half == 0 ? rp : cp;
                const int* idx = half == 0 ? ci : ri;
                const float* val = reinterpret_cast<const float*>(half == 0 ? vt : vct);
                const float4* src4 = reinterpret_cast<const float4*>(half == 0 ? mu_b : nu_b);
                float4* dst4 = reinterpret_cast<float4*>(half == 0 ? a : b);
                const float4* kin4 = reinterpret_cast<const float4*>(half == 0 ? kbB : kbA);
                float4* kout4 = reinterpret_cast<float4*>(half == 0 ? kbA : kbB);
                const float4* Kn4 = half == 0 ? Ks4 : KsT4;    // a -> KA (rows K'[w][.]); b -> KB (rows K'[.][w])
                // four items per step (the same g, so each K' load feeds all four)
                constexpr int IPS = 4;
                for (int jt = 0; jt < n_iter; jt += IPS) {
                    const int g = threadIdx.x % q4;                // it % q4 for every item
                    float4 xv[IPS], s[IPS];
#pragma unroll
                    for (int q = 0; q < IPS; ++q) {
                        const int it = threadIdx.x + (jt + q) * blockDim.x;
                        xv[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                        s[q] = xv[q];
                        if (it < n_items) {
                            xv[q] = primalk_update(it / q4, g, q4, ptr, idx, val, kin4, src4[it]);
                            dst4[it] = xv[q];
                        }
                    }
                    // the block rows sit in lanes lane - g .. lane - g + q4 - 1 (rows
                    // never straddle the valid / invalid boundary: n_items = M q4)
                    const int row0 = lane - g;
                    for (int w4 = 0; w4 < q4; ++w4) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float4 kv = Kn4[(4 * w4 + j) * q4 + g];
#pragma unroll
                            for (int q = 0; q < IPS; ++q) {
                                const float xs = j == 0 ? xv[q].x : j == 1 ? xv[q].y : j == 2 ? xv[q].z : xv[q].w;
                                const float x = __shfl_sync(0xffffffffu, xs, row0 + w4);
                                s[q].x = fmaf(kv.x, x, s[q].x);
                                s[q].y = fmaf(kv.y, x, s[q].y);
                                s[q].z = fmaf(kv.z, x, s[q].z);
                                s[q].w = fmaf(kv.w, x, s[q].w);
                            }
                        }
                    }
#pragma unroll
                    for (int q = 0; q < IPS; ++q) {
                        const int it = threadIdx.x + (jt + q) * blockDim.x;
                        if (it < n_items) kout4[it] = s[q];
                    }
                }
                __syncthreads();
            }
        }
    } else {
        T* kb = kbB;
        for (int sweep = 0; sweep < P.sweeps; ++sweep) {
            for (int half = 0; half < 2; ++half) {
                const T* x = half == 0 ? b : a;
                const T* Kx = half == 0 ? KsT : Ks;
                for (int t = threadIdx.x; t < m; t += blockDim.x) {
                    const int l = t / kk, u = t - (t / kk) * kk;
                    const T* kc = Kx + u;
                    const T* xr = x + l * kk;
                    T acc = T(0);
                    for (int w = 0; w < kk; ++w) acc += kc[w * kk] * xr[w];
                    kb[t] = acc;
                }
                __syncthreads();
                const int* ptr = half == 0 ? rp : cp;
                const int* idx = half == 0 ? ci : ri;
                const T* val = half == 0 ? vt : vct;
                const T* src = half == 0 ? mu_b : nu_b;
                T* dst = half == 0 ? a : b;
                for (int t = threadIdx.x; t < m; t += blockDim.x) {
                    const int k = t / kk, u = t - (t / kk) * kk;
                    T r = T(0);
                    for (int e = ptr[k]; e < ptr[k + 1]; ++e) r += val[e] * kb[idx[e] * kk + u];
                    dst[t] = r > T(0) ? src[t] / r : T(0);
                }
                __syncthreads();
            }
        }
    }
    if (P.a_out || P.b_out)
        for (int t = threadIdx.x; t < m; t += blockDim.x) {
            const int i = blk_pixel(t / kk, t - (t / kk) * kk, n, kap, N);
            if (P.a_out) P.a_out[i] = widen_f32(a[t]);
            if (P.b_out) P.b_out[i] = widen_f32(b[t]);
        }
    // sweeps_only: the evaluation runs spread over many CTAs (primalk_eval_*
    // kernels); a, b stay block-major for them
    if (sweeps_only) return;
    // ---- certified evaluation -----------------------------------------------
    // Per side: each marginal entry mu-hat_i (nu-hat_i) is evaluated as
    // h_i = x_i sum_e pi~_e kd_e, kd = sum_w K' x' (non-negative terms), with
    // |mu-hat_i - h_i| <= rel h_i + slack.  FP64: kd by FP64 fused
    // multiply-adds; FP32 scalings: kd by the compensated dot product Dot2 of
    // Ogita, Rump and Oishi (Accurate sum and dot product, SIAM J. Sci.
    // Comput. 26, 2005; error-free products and sums, kept as hi + lo), within
    // a relative 2 gamma_(2kk)^2 (gamma_n = n u / (1 - n u), u = 2^-24) plus an
    // absolute kk 2^-140 (FP32 underflow).  The gather and the product by x_i
    // add deg + 2 FP64 roundings (deg: the plan's largest row or column
    // degree), a relative (deg + 3) 2^-52 (Higham, Accuracy and Stability of
    // Numerical Algorithms, Sec. 3.1); 2^-1000 covers FP64 underflow.
    // From them: the total mass s within S_h (1 +- (rel + gamma_h)) +- m slack
    // (S_h the round-to-nearest sum of the h_i, gamma_h its summation bound),
    // the s-free sums
    // A = sum_i w_i |mu-hat_i - mu_i| <= sum_i w_i (|h_i - mu_i| + rel h_i)
    // + slack sum_i w_i and B = sum_i w_i mu_i (the SumPool pass's per-block
    // bounds), and sum_i w_i |mu-hat_i / s - mu_i| <= A / s + B |1 / s - 1|.
    int deg = 0;
    for (int q = threadIdx.x; q < M; q += blockDim.x) deg = max(deg, max(rp[q + 1] - rp[q], cp[q + 1] - cp[q]));
    for (int o = 16; o > 0; o >>= 1) deg = max(deg, __shfl_xor_sync(0xffffffffu, deg, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)deg;
    __syncthreads();
    if (threadIdx.x == 0) {
        double d = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) d = fmax(d, red[w]);
        red[32] = d;
    }
    __syncthreads();
    deg = (int)red[32];
    __syncthreads();
    double rel;                                               // relative enclosure of each entry
    double kd_abs;                                            // absolute enclosure of each kd
    if (sizeof(T) == 4) {
        const double g2 = (2.0 * kk * 0x1p-24) / (1.0 - 2.0 * kk * 0x1p-24);
        rel = __dadd_ru(__dmul_ru(2.0, __dmul_ru(g2, g2)), (double)(deg + 3) * 0x1p-52);
        kd_abs = (double)kk * 0x1p-140;
    } else {
        rel = (double)(kk + deg + 3) * 0x1p-52;
        kd_abs = 0.0;
    }
    // the round-to-nearest sum S_h: each h_i meets at most m / blockDim + 40
    // additions (per thread, warp shuffles, warps), Higham Sec. 4.2
    const double gam_m = (double)((m + blockDim.x - 1) / blockDim.x + 42) * 0x1p-52;
    const double w_sum_hi = __dmul_ru((double)m, tv_weight_hi(0, 0, N, P.p));   // >= sum_i w_i (corner = max)
    double* kd = P.kscratch;                                  // m, block-major (mu_b, nu_b are done)
    double s_lo = 0.0, s_hi = HUGE_VAL, A_mu = 0.0, A_nu = 0.0, B_mu = 0.0, B_nu = 0.0, res = 0.0;
    for (int side = 0; side < 2; ++side) {
        // side 0: mu-hat[k, u] = a[k, u] sum_l pi~_kl sum_w K'[u, w] b[l, w]
        // side 1: nu-hat[l, v] = b[l, v] sum_k pi~_kl sum_w K'[w, v] a[k, w]
        const T* oth = side == 0 ? b : a;
        const T* own = side == 0 ? a : b;
        const T* Kx = side == 0 ? KsT : Ks;                   // row w over the output offsets
        if (sizeof(T) == 4 && (kk & 3) == 0) {
            const float4* K4 = reinterpret_cast<const float4*>(Kx);
            for (int it = threadIdx.x; it < (m >> 2); it += blockDim.x) {
                const int l = it / q4, g = it - (it / q4) * q4;
                const float* xr = reinterpret_cast<const float*>(oth) + (size_t)l * kk;
                float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
                for (int w = 0; w < kk; ++w) {
                    const float x = xr[w];
                    const float4 kv = K4[w * q4 + g];
                    const float kc[4] = {kv.x, kv.y, kv.z, kv.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float pr = kc[j] * x;
                        const float pe = fmaf(kc[j], x, -pr);
                        float s, t;
                        two_sum_f(hi[j], pr, s, t);
                        hi[j] = s;
                        lo[j] += t + pe;
                    }
                }
                double2* o2 = reinterpret_cast<double2*>(kd) + 2 * it;
                o2[0] = make_double2(widen_f32(hi[0]) + widen_f32(lo[0]), widen_f32(hi[1]) + widen_f32(lo[1]));
                o2[1] = make_double2(widen_f32(hi[2]) + widen_f32(lo[2]), widen_f32(hi[3]) + widen_f32(lo[3]));
            }
        } else {
            for (int t = threadIdx.x; t < m; t += blockDim.x) {
                const int l = t / kk, u = t - (t / kk) * kk;
                const T* xr = oth + (size_t)l * kk;
                double s = 0.0;
                for (int w = 0; w < kk; ++w) s = fma(widen_f32(Kx[w * kk + u]), widen_f32(xr[w]), s);
                kd[t] = s;
            }
        }
        __syncthreads();
        const int* ptr = side == 0 ? rp : cp;
        const int* idx = side == 0 ? ci : ri;
        const double* val = side == 0 ? P.val : P.valc;
        const double* meas = side == 0 ? P.mu : P.nu;
        double acc_h = 0.0, acc_A = 0.0, acc_res = 0.0, x_max = 0.0;
        for (int t = threadIdx.x; t < m; t += blockDim.x) {
            const int k = t / kk, u = t - (t / kk) * kk;
            double r = 0.0;
            for (int e = ptr[k]; e < ptr[k + 1]; ++e) r = fma(val[e], kd[idx[e] * kk + u], r);
            const double x = widen_f32(own[t]);
            const double h = x * r;
            acc_h += h;
            x_max = fmax(x_max, x);
            const int i = blk_pixel(k, u, n, kap, N);
            const double mi = meas[i];
            const double dmax = fmax(__dsub_ru(h, mi), __dsub_ru(mi, h));      // >= |h - mu_i|
            acc_A = __fma_ru(tv_weight_hi_fast(i / N, i - (i / N) * N, N, P.p), __fma_ru(h, rel, dmax), acc_A);
            acc_res += dmax;
        }
        const double S_h = block_reduce_rn(acc_h, red);
        double A = block_reduce_ru(acc_A, red);
        res += block_reduce_rn(acc_res, red);
        // x_max: block maximum (the kd slack reaches h through sum_e pi~_e <= 1)
        for (int o = 16; o > 0; o >>= 1) x_max = fmax(x_max, __shfl_xor_sync(0xffffffffu, x_max, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x_max;
        __syncthreads();
        if (threadIdx.x == 0) {
            double d = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) d = fmax(d, red[w]);
            red[32] = d;
        }
        __syncthreads();
        const double slack = __dadd_ru(__dmul_ru(red[32], kd_abs), 0x1p-1000);
        __syncthreads();
        A = __fma_ru(slack, w_sum_hi, A);
        const double ms = __dmul_ru((double)m, slack);
        const double rg = __dadd_ru(rel, gam_m);
        // both sides enclose the same total mass s: intersect
        s_lo = fmax(s_lo, __dsub_rd(__dmul_rd(S_h, __dsub_rd(1.0, rg)), ms));
        s_hi = fmin(s_hi, __dadd_ru(__dmul_ru(S_h, __dadd_ru(1.0, rg)), ms));
        // B from the SumPool pass's per-block bounds of sum_{i in block} w_i mu_i
        const double* wb = side == 0 ? P.mu_w_hi : P.nu_w_hi;
        double accB = 0.0;
        for (int q = threadIdx.x; q < M; q += blockDim.x) accB = __dadd_ru(accB, wb[q]);
        const double B = block_reduce_ru(accB, red);
        if (side == 0) { A_mu = A; B_mu = B; } else { A_nu = A; B_nu = B; }
        __syncthreads();                                      // kd is rewritten by the next side
    }
    // ---- cost of the fitted plan over its support, rounded up ---------------
    // position (k, u) of the source, then every plan entry e = (k, l) of its row:
    //   a[k, u] sum_v K'[u, v] b[l, v] rho(x_(k,u), y_(l,v))^p in T rounded up
    //   (K', a, b are exact in T), weighted by pi~_kl in FP64 rounded up
    const T* tab = reinterpret_cast<const T*>(P.ctab_hi);
    double cost = 0.0;
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        const int k = t / kk, u = t - (t / kk) * kk;
        const T a_ku = a[t];
        const T* kh = KsT + u;                                // K'[u][v] = KsT[v kk + u]: lanes on u, no conflicts
        for (int e = rp[k]; e < rp[k + 1]; ++e) {
            const int l = ci[e];
            const int r0 = kap * (k / n - l / n) + u / kap, c0 = kap * (k % n - l % n) + u % kap;
            const T* br = b + l * kk;
            T inner = T(0);
            for (int v1 = 0; v1 < kap; ++v1) {
                const T* trow = tab + abs(r0 - v1) * N;
                for (int v2 = 0; v2 < kap; ++v2) {
                    const int v = v1 * kap + v2;
                    inner = fma_ru(mul_ru(kh[v * kk], br[v]), trow[abs(c0 - v2)], inner);
                }
            }
            cost = __fma_ru(v64[e], widen_f32(mul_ru(a_ku, inner)), cost);
        }
    }
    const double cost_sum = block_reduce_ru(cost, red);
    if (threadIdx.x == 0) {
        const double p = P.p;
        const double inv_hi = s_lo > 0.0 ? __drcp_ru(s_lo) : HUGE_VAL;   // >= 1 / s
        const double inv_lo = __drcp_rd(s_hi);                          // <= 1 / s
        const double dinv = fmax(0.0, fmax(__dsub_ru(inv_hi, 1.0), __dsub_ru(1.0, inv_lo)));
        const double tv_mu = __fma_ru(B_mu, dinv, __dmul_ru(A_mu, inv_hi));
        const double tv_nu = __fma_ru(B_nu, dinv, __dmul_ru(A_nu, inv_hi));
        const double scale = (p == 1.0) ? 1.0 : (p == 2.0 ? 2.0 : __dmul_ru(pow(2.0, p - 1.0), 1.0 + 0x1p-49));
        const double dmu = root_p_ru(__dmul_ru(scale, tv_mu), p);
        const double dnu = root_p_ru(__dmul_ru(scale, tv_nu), p);
        const double w_hat_p = __dmul_ru(cost_sum, inv_hi);
        const double w_hat = root_p_ru(w_hat_p, p);
        PairOut& O = outs[P.out_index];
        O.w_hat_p = w_hat_p;
        O.delta_mu = dmu;
        O.delta_nu = dnu;
        O.ub_primal = __dadd_ru(__dadd_ru(w_hat, dmu), dnu);
        O.ipf_residual = res;
        O.sweeps_done = P.sweeps;
    }
    // leave a, b in the pixel layout of the other passes (through the KB scratch)
    T* tmp = reinterpret_cast<T*>(P.kb_t);
    for (int side = 0; side < 2; ++side) {
        T* x = side == 0 ? a : b;
        for (int t = threadIdx.x; t < m; t += blockDim.x) tmp[t] = x[t];
        __syncthreads();
        for (int t = threadIdx.x; t < m; t += blockDim.x) x[blk_pixel(t / kk, t - (t / kk) * kk, n, kap, N)] = tmp[t];
        __syncthreads();
    }
}

int launch_primalk(const PairDev* pairs_d, PairOut* outs_d, const int* pair_ids, int n_pairs, int kappa_max,
                   int M_max, int nnz_max, int m_max, bool all_kappa4, bool f64, cudaStream_t stream,
                   int sweeps_only) {
    if (n_pairs <= 0) return QWB_OK;
    if (kappa_max > 8) return QWB_ERR_UNSUPPORTED;
    const size_t tsz = f64 ? 8 : 4;
    const int kk = kappa_max * kappa_max;
    const size_t kq = (size_t)kk * kk;
    const size_t base = 2 * align16(tsz * kq);                // K' in two orientations
    // KB and KA in shared memory when they fit; the plan staged as well when
    // it fits next to them
    const size_t kbb = 2 * align16(tsz * (size_t)m_max);
    const bool kb_in = base + kbb <= 200 * 1024;
    const size_t with_kb = kb_in ? base + kbb : base;
    const int cap = std::max(nnz_max, 2 * M_max);
    const size_t csr = (8 + 2 * tsz + 2 * sizeof(int)) * (size_t)cap + 2 * sizeof(int) * (size_t)(M_max + 1);
    const bool staged = with_kb + csr <= 220 * 1024;
    const size_t smem = staged ? with_kb + csr : with_kb;
    const int csr_cap = staged ? cap : -1;
    const int kb_cap = kb_in ? m_max : 0;
    const int threads = f64 ? PRIMALK_THREADS_F64 : PRIMALK_THREADS_F32;
    auto run = [&](auto kern) -> int {
        QWB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<n_pairs, threads, smem, stream>>>(pairs_d, outs_d, pair_ids, csr_cap, kk, kb_cap, sweeps_only);
        QWB_LAUNCHED();
        return QWB_OK;
    };
    if (f64) return all_kappa4 ? run(primalk_kernel<double, 16>) : run(primalk_kernel<double, 0>);
    return all_kappa4 ? run(primalk_kernel<float, 16>) : run(primalk_kernel<float, 0>);
}

// --------------------------------------------------------------------------
// primalk_cl: the primal pass of primalk_kernel (the same definition, the
// same fine sweeps item for item, the same certified evaluation) for FP32
// pairs with kappa 2, 4 or 8, one pair on a thread-block cluster of C CTAs.
// CTA `rank` owns the block rows [rank R, (rank + 1) R), R = ceil(n / C):
// blocks [k0, k0 + nb) and, because whole block rows are owned, the same
// range of positions in the block-major and in the pixel layout.  It keeps
// the KB rows of its own target blocks and the KA rows of its own source
// blocks in shared memory; a half sweep reads the other CTAs' rows through
// distributed shared memory and ends at a cluster barrier (KB and KA are
// separate buffers, so one barrier per half suffices).  The evaluation runs
// on the owned blocks as well: the kd rows of both sides go to global memory
// (cluster barrier), each CTA gathers the marginal entries of its rows and
// columns and its part of the support cost, and rank 0 combines the CTAs'
// partial sums, read from their shared memory, into the bounds.  With
// several CTAs per pair, a batch of pairs spreads over all SMs in one wave
// instead of one CTA per SM in two.
//   Enclosures: as in primalk_kernel, with two changes that only tighten
// them.  The total mass is enclosed by a round-down and a round-up sum of
// the h_i (no summation bound needed), and |h_i - mu_i| is taken from the
// nearest-rounded difference d_i, |h_i - mu_i| <= |d_i| + 2^-53 (h_i + mu_i),
// so sum_i w_i |mu-hat_i - mu_i| <= sum w |d| + (rel + 2^-53) sum w h
// + 2^-53 B + slack sum w, every sum rounded up.
// --------------------------------------------------------------------------
constexpr int PKC_PARTS = 16;

__device__ __forceinline__ double block_reduce_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s = fmax(s, red[w]);
        red[32] = s;
    }
    __syncthreads();
    return red[32];
}

template <int KK, int TH, int MINB>
__global__ void __launch_bounds__(TH, MINB)
primalk_cl_kernel(const PairDev* __restrict__ pairs, PairOut* __restrict__ outs,
                  const int* __restrict__ pair_ids, int C, int kb_cap, int csr_cap) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[33];
    __shared__ double part[PKC_PARTS];
    constexpr int q4 = KK / 4;                                // float4s per block row
    constexpr int IPS = 4;                                    // items per step (one K' load feeds four)
    static_assert(TH % q4 == 0 && 32 % q4 == 0, "a block row lies in one warp");
    const int rank = (int)cl.block_rank();
    const PairDev& P = pairs[pair_ids[blockIdx.x / C]];
    const int N = P.N, kap = P.kappa, n = P.n, m = P.m;
    const int R = (n + C - 1) / C, Rn = R * n;                // block rows and blocks per CTA
    const int r0 = min(n, rank * R), r1 = min(n, r0 + R);
    const int k0 = r0 * n, nb = (r1 - r0) * n;                // owned blocks [k0, k0 + nb)
    const int t0 = k0 * KK, tn = nb * KK;                     // owned positions
    float* Ks = reinterpret_cast<float*>(smem_raw);           // row w: K'[w][.]
    float* KsT = Ks + KK * KK;                                // row w: K'[.][w]
    float* kbB = KsT + KK * KK;                               // KB rows of the owned blocks
    float* kbA = kbB + kb_cap;                                // KA rows of the owned blocks
    // the plan's rows of the owned source blocks and columns of the owned
    // target blocks, staged with offsets relative to the first owned entry
    // (when they fit csr_cap; else read from global memory)
    float* v_s = kbA + kb_cap;
    float* vc_s = v_s + csr_cap;
    int* ci_s = reinterpret_cast<int*>(vc_s + csr_cap);
    int* ri_s = ci_s + csr_cap;
    int* rp_s = ri_s + csr_cap;                               // Rn + 1 entries each
    int* cp_s = rp_s + Rn + 1;
    for (int t = threadIdx.x; t < KK * KK; t += TH) {
        const int u = t / KK, w = t - u * KK;
        const float kt = reinterpret_cast<const float*>(P.upK_t)[t];
        Ks[t] = kt;
        KsT[w * KK + u] = kt;
    }
    const int r_base = P.rowptr[k0], c_base = P.colptr[k0];
    const int r_cnt = P.rowptr[k0 + nb] - r_base, c_cnt = P.colptr[k0 + nb] - c_base;
    const bool staged = r_cnt <= csr_cap && c_cnt <= csr_cap;
    if (staged) {
        for (int q = threadIdx.x; q <= nb; q += TH) {
            rp_s[q] = P.rowptr[k0 + q] - r_base;
            cp_s[q] = P.colptr[k0 + q] - c_base;
        }
        const float* vt = reinterpret_cast<const float*>(P.val_t);
        const float* vct = reinterpret_cast<const float*>(P.valc_t);
        for (int e = threadIdx.x; e < r_cnt; e += TH) { ci_s[e] = P.colidx[r_base + e]; v_s[e] = vt[r_base + e]; }
        for (int e = threadIdx.x; e < c_cnt; e += TH) { ri_s[e] = P.rowidx[c_base + e]; vc_s[e] = vct[c_base + e]; }
    }
    float* a = reinterpret_cast<float*>(P.a);
    float* b = reinterpret_cast<float*>(P.b);
    float* mu_b = reinterpret_cast<float*>(P.kscratch);       // block-major mu, nu (sweeps only)
    float* nu_b = mu_b + m;
    const float* mu_t = reinterpret_cast<const float*>(P.mu_t);
    const float* nu_t = reinterpret_cast<const float*>(P.nu_t);
    for (int t = threadIdx.x; t < tn; t += TH) {
        const int tt = t0 + t;
        const int i = blk_pixel(tt / KK, tt - (tt / KK) * KK, n, kap, N);
        mu_b[tt] = mu_t[i];
        nu_b[tt] = nu_t[i];
        b[tt] = 1.0f;
    }
    __syncthreads();
    const float4* Ks4 = reinterpret_cast<const float4*>(Ks);
    const float4* KsT4 = reinterpret_cast<const float4*>(KsT);
    const int n_own = nb * q4;                                // float4 items of the owned blocks
    const int n_iter = (n_own + TH - 1) / TH;                 // the same for every thread of the CTA
    const int g = threadIdx.x % q4;                           // item % q4 for every item of the thread
    const int row0 = (threadIdx.x & 31) - g;                  // first lane of the item's block row
    // b = 1: KB[l, u] = sum_w K'[u][w]
    for (int it = threadIdx.x; it < n_own; it += TH) {
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int w = 0; w < KK; ++w) {
            const float4 kv = KsT4[w * q4 + g];
            s.x += kv.x; s.y += kv.y; s.z += kv.z; s.w += kv.w;
        }
        reinterpret_cast<float4*>(kbB)[it] = s;
    }
    cl.sync();                                                // KB rows visible to the cluster
    for (int sweep = 0; sweep < P.sweeps; ++sweep) {
        for (int half = 0; half < 2; ++half) {
            // owned row (column) kl: entries [ptr[kl], ptr[kl + 1]) of idx / val
            const int* ptr = staged ? (half == 0 ? rp_s : cp_s) : (half == 0 ? P.rowptr + k0 : P.colptr + k0);
            const int* idx = staged ? (half == 0 ? ci_s : ri_s) : (half == 0 ? P.colidx : P.rowidx);
            const float* val = staged ? (half == 0 ? v_s : vc_s)
                                      : reinterpret_cast<const float*>(half == 0 ? P.val_t : P.valc_t);
            const float4* src4 = reinterpret_cast<const float4*>(half == 0 ? mu_b : nu_b) + k0 * q4;
            float4* dst4 = reinterpret_cast<float4*>(half == 0 ? a : b) + k0 * q4;
            float* kin = half == 0 ? kbB : kbA;               // this CTA's rows; the others' by rank
            float4* kout4 = reinterpret_cast<float4*>(half == 0 ? kbA : kbB);
            const float4* Kn4 = half == 0 ? Ks4 : KsT4;       // a -> KA (rows K'[w][.]); b -> KB
            for (int jt = 0; jt < n_iter; jt += IPS) {
                float4 xv[IPS], s[IPS], sv[IPS], r[IPS];
                int e0[IPS], e1[IPS];
                int dmax = 0;
                // the items' measure values and plan ranges first, then their
                // gathers side by side (each item's terms in entry order)
#pragma unroll
                for (int q = 0; q < IPS; ++q) {
                    const int it = threadIdx.x + (jt + q) * TH;
                    s[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                    r[q] = s[q];
                    sv[q] = s[q];
                    e0[q] = e1[q] = 0;
                    if (it < n_own) {
                        sv[q] = src4[it];
                        e0[q] = ptr[it / q4];
                        e1[q] = ptr[it / q4 + 1];
                        dmax = max(dmax, e1[q] - e0[q]);
                    }
                }
                for (int d = 0; d < dmax; ++d) {
#pragma unroll
                    for (int q = 0; q < IPS; ++q) {
                        const int e = e0[q] + d;
                        if (e < e1[q]) {
                            const int l = idx[e], owner = l / Rn;
                            const float4* peer = reinterpret_cast<const float4*>(cl.map_shared_rank(kin, owner));
                            const float4 kv = peer[(l - owner * Rn) * q4 + g];
                            const float v = val[e];
                            r[q].x = fmaf(v, kv.x, r[q].x);
                            r[q].y = fmaf(v, kv.y, r[q].y);
                            r[q].z = fmaf(v, kv.z, r[q].z);
                            r[q].w = fmaf(v, kv.w, r[q].w);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < IPS; ++q) {
                    const int it = threadIdx.x + (jt + q) * TH;
                    xv[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (it < n_own) {
                        xv[q] = make_float4(ipf_div(sv[q].x, r[q].x), ipf_div(sv[q].y, r[q].y),
                                            ipf_div(sv[q].z, r[q].z), ipf_div(sv[q].w, r[q].w));
                        dst4[it] = xv[q];
                    }
                }
                for (int w4 = 0; w4 < q4; ++w4) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float4 kv = Kn4[(4 * w4 + j) * q4 + g];
#pragma unroll
                        for (int q = 0; q < IPS; ++q) {
                            const float xs = j == 0 ? xv[q].x : j == 1 ? xv[q].y : j == 2 ? xv[q].z : xv[q].w;
                            const float x = __shfl_sync(0xffffffffu, xs, row0 + w4);
                            s[q].x = fmaf(kv.x, x, s[q].x);
                            s[q].y = fmaf(kv.y, x, s[q].y);
                            s[q].z = fmaf(kv.z, x, s[q].z);
                            s[q].w = fmaf(kv.w, x, s[q].w);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < IPS; ++q) {
                    const int it = threadIdx.x + (jt + q) * TH;
                    if (it < n_own) kout4[it] = s[q];
                }
            }
            cl.sync();                                        // the next half reads the new rows
        }
    }
    if (P.a_out || P.b_out)
        for (int t = threadIdx.x; t < tn; t += TH) {
            const int tt = t0 + t;
            const int i = blk_pixel(tt / KK, tt - (tt / KK) * KK, n, kap, N);
            if (P.a_out) P.a_out[i] = widen_f32(a[tt]);
            if (P.b_out) P.b_out[i] = widen_f32(b[tt]);
        }
    // ---- certified evaluation on the owned blocks ---------------------------
    // kd rows of both sides: side 0 (mu-hat) kd[l, u] = sum_w K'[u, w] b[l, w]
    // for the owned l, side 1 (nu-hat) kd[k, v] = sum_w K'[w, v] a[k, w] for
    // the owned k, by the compensated dot product Dot2 in FP32 (hi + lo)
    double* kd0 = P.kscratch;                                 // mu_b, nu_b are done (last barrier)
    double* kd1 = P.kscratch + m;
    for (int side = 0; side < 2; ++side) {
        const float* oth = side == 0 ? b : a;
        const float4* K4 = side == 0 ? KsT4 : Ks4;            // row w over the output offsets
        double2* kd2 = reinterpret_cast<double2*>(side == 0 ? kd0 : kd1);
        for (int it = threadIdx.x; it < n_own; it += TH) {
            const int git = k0 * q4 + it;
            const float* xr = oth + (size_t)(git / q4) * KK;
            float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
            for (int w = 0; w < KK; ++w) {
                const float x = xr[w];
                const float4 kv = K4[w * q4 + g];
                const float kc[4] = {kv.x, kv.y, kv.z, kv.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float pr = kc[j] * x;
                    const float pe = fmaf(kc[j], x, -pr);
                    float s, t;
                    two_sum_f(hi[j], pr, s, t);
                    hi[j] = s;
                    lo[j] += t + pe;
                }
            }
            kd2[2 * git] = make_double2(widen_f32(hi[0]) + widen_f32(lo[0]), widen_f32(hi[1]) + widen_f32(lo[1]));
            kd2[2 * git + 1] = make_double2(widen_f32(hi[2]) + widen_f32(lo[2]), widen_f32(hi[3]) + widen_f32(lo[3]));
        }
    }
    // the owned rows (side 0) and columns (side 1) of the plan: local index
    // kl = k - k0, entries [ptr[kl], ptr[kl + 1]) of idx and of the FP64 values
    const int* ptr_s[2] = {staged ? rp_s : P.rowptr + k0, staged ? cp_s : P.colptr + k0};
    const int* idx_s[2] = {staged ? ci_s : P.colidx, staged ? ri_s : P.rowidx};
    const double* v64_s[2] = {staged ? P.val + r_base : P.val, staged ? P.valc + c_base : P.valc};
    int deg = 0;                                              // largest row / column degree (owned)
    for (int q = threadIdx.x; q < nb; q += TH)
        deg = max(deg, max(ptr_s[0][q + 1] - ptr_s[0][q], ptr_s[1][q + 1] - ptr_s[1][q]));
    const double deg_cta = block_reduce_max((double)deg, red);
    cl.sync();                                                // every CTA's kd rows visible
    // marginal entries of the owned rows (side 0) and columns (side 1):
    // h = x r with r = sum_e pi~_e kd[idx_e, u] (FP64 FMAs), x the own scaling
    double sums[12];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int* ptr = ptr_s[side];
        const int* idx = idx_s[side];
        const double* val = v64_s[side];
        const double* meas = side == 0 ? P.mu : P.nu;
        const float* own = side == 0 ? a : b;
        const double* kd = side == 0 ? kd0 : kd1;
        double s_lo = 0.0, s_hi = 0.0, dsum = 0.0, whsum = 0.0, rsum = 0.0;
        float xm = 0.0f;
        for (int t = threadIdx.x; t < tn; t += TH) {
            const int tt = t0 + t;
            const int k = tt / KK, u = tt - (tt / KK) * KK;
            double r = 0.0;
            for (int e = ptr[k - k0]; e < ptr[k - k0 + 1]; ++e) r = fma(val[e], kd[idx[e] * KK + u], r);
            const float xf = own[tt];
            const double h = widen_f32(xf) * r;
            s_lo = __dadd_rd(s_lo, h);
            s_hi = __dadd_ru(s_hi, h);
            const int i = blk_pixel(k, u, n, kap, N);
            const double ad = fabs(h - meas[i]);              // nearest-rounded |h - mu_i|
            const double w = tv_weight_hi_fast(i / N, i - (i / N) * N, N, P.p);
            dsum = __fma_ru(w, ad, dsum);
            whsum = __fma_ru(w, h, whsum);
            rsum += ad;
            xm = fmaxf(xm, xf);
        }
        sums[6 * side + 0] = block_reduce_rd(s_lo, red);
        sums[6 * side + 1] = block_reduce_ru(s_hi, red);
        sums[6 * side + 2] = block_reduce_ru(dsum, red);
        sums[6 * side + 3] = block_reduce_ru(whsum, red);
        sums[6 * side + 4] = block_reduce_rn(rsum, red);
        sums[6 * side + 5] = block_reduce_max(widen_f32(xm), red);
    }
    // B: the SumPool pass's per-block bounds of sum_{i in block} w_i mu_i (owned blocks)
    double bmu = 0.0, bnu = 0.0;
    for (int q = threadIdx.x; q < nb; q += TH) {
        bmu = __dadd_ru(bmu, P.mu_w_hi[k0 + q]);
        bnu = __dadd_ru(bnu, P.nu_w_hi[k0 + q]);
    }
    const double B_mu_cta = block_reduce_ru(bmu, red);
    const double B_nu_cta = block_reduce_ru(bnu, red);
    // cost of the fitted plan over its support (owned source positions), as primalk_kernel
    const float* tab = reinterpret_cast<const float*>(P.ctab_hi);
    double cost = 0.0;
    for (int t = threadIdx.x; t < tn; t += TH) {
        const int tt = t0 + t;
        const int k = tt / KK, u = tt - (tt / KK) * KK;
        const float a_ku = a[tt];
        const float* kh = KsT + u;                            // K'[u][v] = KsT[v KK + u]
        for (int e = ptr_s[0][k - k0]; e < ptr_s[0][k - k0 + 1]; ++e) {
            const int l = idx_s[0][e];
            const int rr = kap * (k / n - l / n) + u / kap, c0 = kap * (k % n - l % n) + u % kap;
            const float* br = b + l * KK;
            float inner = 0.0f;
            for (int v1 = 0; v1 < kap; ++v1) {
                const float* trow = tab + abs(rr - v1) * N;
                for (int v2 = 0; v2 < kap; ++v2) {
                    const int v = v1 * kap + v2;
                    inner = fma_ru(mul_ru(kh[v * KK], br[v]), trow[abs(c0 - v2)], inner);
                }
            }
            cost = __fma_ru(v64_s[0][e], widen_f32(mul_ru(a_ku, inner)), cost);
        }
    }
    const double cost_cta = block_reduce_ru(cost, red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < 12; ++q) part[q] = sums[q];
        part[12] = B_mu_cta;
        part[13] = B_nu_cta;
        part[14] = cost_cta;
        part[15] = deg_cta;
    }
    cl.sync();                                                // partials published; b no longer read
    if (rank == 0 && threadIdx.x == 0) {
        double tot[PKC_PARTS];
#pragma unroll
        for (int q = 0; q < PKC_PARTS; ++q) tot[q] = 0.0;
        for (int r = 0; r < C; ++r) {
            const double* pr = cl.map_shared_rank(part, r);
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int o = 6 * side;
                tot[o + 0] = __dadd_rd(tot[o + 0], pr[o + 0]);
                tot[o + 1] = __dadd_ru(tot[o + 1], pr[o + 1]);
                tot[o + 2] = __dadd_ru(tot[o + 2], pr[o + 2]);
                tot[o + 3] = __dadd_ru(tot[o + 3], pr[o + 3]);
                tot[o + 4] += pr[o + 4];
                tot[o + 5] = fmax(tot[o + 5], pr[o + 5]);
            }
            tot[12] = __dadd_ru(tot[12], pr[12]);
            tot[13] = __dadd_ru(tot[13], pr[13]);
            tot[14] = __dadd_ru(tot[14], pr[14]);
            tot[15] = fmax(tot[15], pr[15]);
        }
        // relative enclosure of each entry (Dot2 in FP32, the gather and the
        // product in FP64) and the absolute one of each kd, as primalk_kernel
        const double g2 = (2.0 * KK * 0x1p-24) / (1.0 - 2.0 * KK * 0x1p-24);
        const double rel = __dadd_ru(__dmul_ru(2.0, __dmul_ru(g2, g2)), (tot[15] + 3.0) * 0x1p-52);
        const double kd_abs = (double)KK * 0x1p-140;
        const double w_sum_hi = __dmul_ru((double)m, tv_weight_hi(0, 0, N, P.p));   // >= sum_i w_i
        const double rel_d = __dadd_ru(rel, 0x1p-53);
        double s_lo = 0.0, s_hi = HUGE_VAL, A[2];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int o = 6 * side;
            const double B = tot[12 + side];
            const double slack = __dadd_ru(__dmul_ru(tot[o + 5], kd_abs), 0x1p-1000);
            double As = __fma_ru(rel_d, tot[o + 3], tot[o + 2]);
            As = __fma_ru(0x1p-53, B, As);
            A[side] = __fma_ru(slack, w_sum_hi, As);
            const double ms = __dmul_ru((double)m, slack);
            s_lo = fmax(s_lo, __dsub_rd(__dmul_rd(tot[o + 0], __dsub_rd(1.0, rel)), ms));
            s_hi = fmin(s_hi, __dadd_ru(__dmul_ru(tot[o + 1], __dadd_ru(1.0, rel)), ms));
        }
        const double p = P.p;
        const double inv_hi = s_lo > 0.0 ? __drcp_ru(s_lo) : HUGE_VAL;   // >= 1 / s
        const double inv_lo = __drcp_rd(s_hi);                          // <= 1 / s
        const double dinv = fmax(0.0, fmax(__dsub_ru(inv_hi, 1.0), __dsub_ru(1.0, inv_lo)));
        const double tv_mu = __fma_ru(tot[12], dinv, __dmul_ru(A[0], inv_hi));
        const double tv_nu = __fma_ru(tot[13], dinv, __dmul_ru(A[1], inv_hi));
        const double scale = (p == 1.0) ? 1.0 : (p == 2.0 ? 2.0 : __dmul_ru(pow(2.0, p - 1.0), 1.0 + 0x1p-49));
        const double dmu = root_p_ru(__dmul_ru(scale, tv_mu), p);
        const double dnu = root_p_ru(__dmul_ru(scale, tv_nu), p);
        const double w_hat_p = __dmul_ru(tot[14], inv_hi);
        PairOut& O = outs[P.out_index];
        O.w_hat_p = w_hat_p;
        O.delta_mu = dmu;
        O.delta_nu = dnu;
        O.ub_primal = __dadd_ru(__dadd_ru(root_p_ru(w_hat_p, p), dmu), dnu);
        O.ipf_residual = tot[4] + tot[10];
        O.sweeps_done = P.sweeps;
    }
    // leave a, b in the pixel layout of the other passes: the owned range maps
    // onto itself, staged through this CTA's KB / KA rows
    for (int side = 0; side < 2; ++side) {
        float* x = side == 0 ? a : b;
        float* tmp = side == 0 ? kbB : kbA;
        for (int t = threadIdx.x; t < tn; t += TH) tmp[t] = x[t0 + t];
        __syncthreads();
        for (int t = threadIdx.x; t < tn; t += TH) {
            const int tt = t0 + t;
            x[blk_pixel(tt / KK, tt - (tt / KK) * KK, n, kap, N)] = tmp[t];
        }
    }
    cl.sync();                                                // rank 0 has read every partial
}

int launch_primalk_cl(const PairDev* pairs_d, PairOut* outs_d, const int* pair_ids, int n_pairs, int kappa,
                      int C, int variant, int n_max, cudaStream_t stream) {
    if (n_pairs <= 0) return QWB_OK;
    if ((kappa != 2 && kappa != 4 && kappa != 8) || C < 1 || C > 8 || variant < 0 || variant > 2)
        return QWB_ERR_UNSUPPORTED;
    const int kk = kappa * kappa;
    const int R = (n_max + C - 1) / C;
    const int kb_cap = R * n_max * kk;                        // floats per KB / KA array
    // staged plan: a basic plan has at most 2M - 1 entries, about 2 per
    // block; room for twice that per CTA (a CTA whose rows hold more reads
    // its part of the plan from global memory)
    const int csr_cap = 4 * R * n_max;
    const size_t smem = sizeof(float) * (2 * (size_t)kk * kk + 2 * (size_t)kb_cap) +
                        (size_t)csr_cap * 2 * (sizeof(float) + sizeof(int)) + 2 * sizeof(int) * (size_t)(R * n_max + 1);
    if (smem + 1024 > 227 * 1024) return QWB_ERR_UNSUPPORTED;   // 1 KB: the kernel's static shared memory
    // variants: threads per CTA and the CTAs per SM the register budget allows
    static const int threads_of[3] = {256, 128, 64};
    auto run = [&](auto kern) -> int {
        QWB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(n_pairs * C));
        cfg.blockDim = dim3((unsigned)threads_of[variant]);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        QWB_CUDA(cudaLaunchKernelEx(&cfg, kern, pairs_d, outs_d, pair_ids, C, kb_cap, csr_cap));
        QWB_LAUNCHED();
        return QWB_OK;
    };
    switch (kk * 4 + variant) {
        case 4 * 4 + 0: return run(primalk_cl_kernel<4, 256, 2>);
        case 4 * 4 + 1: return run(primalk_cl_kernel<4, 128, 5>);
        case 4 * 4 + 2: return run(primalk_cl_kernel<4, 64, 10>);
        case 16 * 4 + 0: return run(primalk_cl_kernel<16, 256, 2>);
        case 16 * 4 + 1: return run(primalk_cl_kernel<16, 128, 5>);
        case 16 * 4 + 2: return run(primalk_cl_kernel<16, 64, 10>);
        case 64 * 4 + 0: return run(primalk_cl_kernel<64, 256, 2>);
        case 64 * 4 + 1: return run(primalk_cl_kernel<64, 128, 5>);
        default: return run(primalk_cl_kernel<64, 64, 10>);
    }
}

// --------------------------------------------------------------------------
// primalk_eval: the certified evaluation of the general-kernel primal pass
// (the enclosures of primalk_cl_kernel) spread over one CTA per (pair,
// coarse block row), after the one-CTA sweeps (primalk_kernel with
// sweeps_only) left a, b block-major.  Four launches: the K products of both
// sides per row (kd, FP64, into the pair's kscratch), the marginal entries,
// the support cost and the TV terms per row (partial sums into the pair's
// kb_t scratch), one combination per pair, then the pixel layout of a, b per
// row (a row's positions map onto themselves).  With many small CTAs the
// FP64 work reaches every SM instead of one SM per pair.
// --------------------------------------------------------------------------
constexpr int PKE_THREADS = 128;

template <int KK>
__global__ void __launch_bounds__(PKE_THREADS)
primalk_eval_kd_kernel(const PairDev* __restrict__ pairs, const int* __restrict__ pair_ids, int n_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int q4 = KK / 4;
    const PairDev& P = pairs[pair_ids[blockIdx.x / n_max]];
    const int k1 = blockIdx.x % n_max, n = P.n, m = P.m;
    if (k1 >= n) return;
    float* Ks = reinterpret_cast<float*>(smem_raw);           // row w: K'[w][.]
    float* KsT = Ks + KK * KK;                                // row w: K'[.][w]
    for (int t = threadIdx.x; t < KK * KK; t += blockDim.x) {
        const int u = t / KK, w = t - u * KK;
        const float kt = reinterpret_cast<const float*>(P.upK_t)[t];
        Ks[t] = kt;
        KsT[w * KK + u] = kt;
    }
    __syncthreads();
    const float* a = reinterpret_cast<const float*>(P.a);
    const float* b = reinterpret_cast<const float*>(P.b);
    const int it0 = k1 * n * q4, n_it = n * q4;                // the row's float4 items
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const float* oth = side == 0 ? b : a;
        const float4* K4 = reinterpret_cast<const float4*>(side == 0 ? KsT : Ks);
        double2* kd2 = reinterpret_cast<double2*>(P.kscratch + (side == 0 ? 0 : m));
        for (int il = threadIdx.x; il < n_it; il += blockDim.x) {
            const int git = it0 + il, g = git % q4;
            const float* xr = oth + (size_t)(git / q4) * KK;
            float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
            for (int w = 0; w < KK; ++w) {
                const float x = xr[w];
                const float4 kv = K4[w * q4 + g];
                const float kc[4] = {kv.x, kv.y, kv.z, kv.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float pr = kc[j] * x;
                    const float pe = fmaf(kc[j], x, -pr);
                    float s, t;
                    two_sum_f(hi[j], pr, s, t);
                    hi[j] = s;
                    lo[j] += t + pe;
                }
            }
            kd2[2 * git] = make_double2(widen_f32(hi[0]) + widen_f32(lo[0]), widen_f32(hi[1]) + widen_f32(lo[1]));
            kd2[2 * git + 1] = make_double2(widen_f32(hi[2]) + widen_f32(lo[2]), widen_f32(hi[3]) + widen_f32(lo[3]));
        }
    }
}

// partial sums per row: [0..5] side 0, [6..11] side 1 (round-down mass, round-up
// mass, sum w |d|, sum w h, residual, largest scaling), B_mu, B_nu, cost, degree
constexpr int PKE_PARTS = 16;

template <int KK>
__global__ void __launch_bounds__(PKE_THREADS)
primalk_eval_sum_kernel(const PairDev* __restrict__ pairs, const int* __restrict__ pair_ids, int n_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[33];
    const PairDev& P = pairs[pair_ids[blockIdx.x / n_max]];
    const int k1 = blockIdx.x % n_max, n = P.n, m = P.m, N = P.N, kap = P.kappa;
    if (k1 >= n) return;
    float* KsT = reinterpret_cast<float*>(smem_raw);          // K'[u][v] = KsT[v KK + u]
    for (int t = threadIdx.x; t < KK * KK; t += blockDim.x) {
        const int u = t / KK, w = t - u * KK;
        KsT[w * KK + u] = reinterpret_cast<const float*>(P.upK_t)[t];
    }
    __syncthreads();
    const float* a = reinterpret_cast<const float*>(P.a);
    const float* b = reinterpret_cast<const float*>(P.b);
    const int k0 = k1 * n, t0 = k0 * KK, tn = n * KK;          // the row's blocks and positions
    int deg = 0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int k = k0 + q;
        deg = max(deg, max(P.rowptr[k + 1] - P.rowptr[k], P.colptr[k + 1] - P.colptr[k]));
    }
    const double deg_row = block_reduce_max((double)deg, red);
    double sums[12];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int* ptr = side == 0 ? P.rowptr : P.colptr;
        const int* idx = side == 0 ? P.colidx : P.rowidx;
        const double* val = side == 0 ? P.val : P.valc;
        const double* meas = side == 0 ? P.mu : P.nu;
        const float* own = side == 0 ? a : b;
        const double* kd = P.kscratch + (side == 0 ? 0 : m);
        double s_lo = 0.0, s_hi = 0.0, dsum = 0.0, whsum = 0.0, rsum = 0.0;
        float xm = 0.0f;
        for (int t = threadIdx.x; t < tn; t += blockDim.x) {
            const int tt = t0 + t;
            const int k = tt / KK, u = tt - (tt / KK) * KK;
            double r = 0.0;
            for (int e = ptr[k]; e < ptr[k + 1]; ++e) r = fma(val[e], kd[idx[e] * KK + u], r);
            const float xf = own[tt];
            const double h = widen_f32(xf) * r;
            s_lo = __dadd_rd(s_lo, h);
            s_hi = __dadd_ru(s_hi, h);
            const int i = blk_pixel(k, u, n, kap, N);
            const double ad = fabs(h - meas[i]);              // nearest-rounded |h - mu_i|
            const double w = tv_weight_hi_fast(i / N, i - (i / N) * N, N, P.p);
            dsum = __fma_ru(w, ad, dsum);
            whsum = __fma_ru(w, h, whsum);
            rsum += ad;
            xm = fmaxf(xm, xf);
        }
        sums[6 * side + 0] = block_reduce_rd(s_lo, red);
        sums[6 * side + 1] = block_reduce_ru(s_hi, red);
        sums[6 * side + 2] = block_reduce_ru(dsum, red);
        sums[6 * side + 3] = block_reduce_ru(whsum, red);
        sums[6 * side + 4] = block_reduce_rn(rsum, red);
        sums[6 * side + 5] = block_reduce_max(widen_f32(xm), red);
    }
    double bmu = 0.0, bnu = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        bmu = __dadd_ru(bmu, P.mu_w_hi[k0 + q]);
        bnu = __dadd_ru(bnu, P.nu_w_hi[k0 + q]);
    }
    const double B_mu_row = block_reduce_ru(bmu, red);
    const double B_nu_row = block_reduce_ru(bnu, red);
    const float* tab = reinterpret_cast<const float*>(P.ctab_hi);
    double cost = 0.0;
    for (int t = threadIdx.x; t < tn; t += blockDim.x) {
        const int tt = t0 + t;
        const int k = tt / KK, u = tt - (tt / KK) * KK;
        const float a_ku = a[tt];
        const float* kh = KsT + u;
        for (int e = P.rowptr[k]; e < P.rowptr[k + 1]; ++e) {
            const int l = P.colidx[e];
            const int rr = kap * (k / n - l / n) + u / kap, c0 = kap * (k % n - l % n) + u % kap;
            const float* br = b + l * KK;
            float inner = 0.0f;
            for (int v1 = 0; v1 < kap; ++v1) {
                const float* trow = tab + abs(rr - v1) * N;
                for (int v2 = 0; v2 < kap; ++v2) {
                    const int v = v1 * kap + v2;
                    inner = fma_ru(mul_ru(kh[v * KK], br[v]), trow[abs(c0 - v2)], inner);
                }
            }
            cost = __fma_ru(P.val[e], widen_f32(mul_ru(a_ku, inner)), cost);
        }
    }
    const double cost_row = block_reduce_ru(cost, red);
    if (threadIdx.x == 0) {
        double* part = reinterpret_cast<double*>(P.kb_t) + (size_t)k1 * PKE_PARTS;
#pragma unroll
        for (int q = 0; q < 12; ++q) part[q] = sums[q];
        part[12] = B_mu_row;
        part[13] = B_nu_row;
        part[14] = cost_row;
        part[15] = deg_row;
    }
}

template <int KK>
__global__ void primalk_eval_final_kernel(const PairDev* __restrict__ pairs, PairOut* __restrict__ outs,
                                          const int* __restrict__ pair_ids) {
    const PairDev& P = pairs[pair_ids[blockIdx.x]];
    if (threadIdx.x != 0) return;
    const int n = P.n, m = P.m, N = P.N;
    double tot[PKE_PARTS];
#pragma unroll
    for (int q = 0; q < PKE_PARTS; ++q) tot[q] = 0.0;
    const double* part = reinterpret_cast<const double*>(P.kb_t);
    for (int r = 0; r < n; ++r) {
        const double* pr = part + (size_t)r * PKE_PARTS;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int o = 6 * side;
            tot[o + 0] = __dadd_rd(tot[o + 0], pr[o + 0]);
            tot[o + 1] = __dadd_ru(tot[o + 1], pr[o + 1]);
            tot[o + 2] = __dadd_ru(tot[o + 2], pr[o + 2]);
            tot[o + 3] = __dadd_ru(tot[o + 3], pr[o + 3]);
            tot[o + 4] += pr[o + 4];
            tot[o + 5] = fmax(tot[o + 5], pr[o + 5]);
        }
        tot[12] = __dadd_ru(tot[12], pr[12]);
        tot[13] = __dadd_ru(tot[13], pr[13]);
        tot[14] = __dadd_ru(tot[14], pr[14]);
        tot[15] = fmax(tot[15], pr[15]);
    }
    // the enclosures of primalk_cl_kernel's combination
    const double g2 = (2.0 * KK * 0x1p-24) / (1.0 - 2.0 * KK * 0x1p-24);
    const double rel = __dadd_ru(__dmul_ru(2.0, __dmul_ru(g2, g2)), (tot[15] + 3.0) * 0x1p-52);
    const double kd_abs = (double)KK * 0x1p-140;
    const double w_sum_hi = __dmul_ru((double)m, tv_weight_hi(0, 0, N, P.p));
    const double rel_d = __dadd_ru(rel, 0x1p-53);
    double s_lo = 0.0, s_hi = HUGE_VAL, A[2];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int o = 6 * side;
        const double B = tot[12 + side];
        const double slack = __dadd_ru(__dmul_ru(tot[o + 5], kd_abs), 0x1p-1000);
        double As = __fma_ru(rel_d, tot[o + 3], tot[o + 2]);
        As = __fma_ru(0x1p-53, B, As);
        A[side] = __fma_ru(slack, w_sum_hi, As);
        const double ms = __dmul_ru((double)m, slack);
        s_lo = fmax(s_lo, __dsub_rd(__dmul_rd(tot[o + 0], __dsub_rd(1.0, rel)), ms));
        s_hi = fmin(s_hi, __dadd_ru(__dmul_ru(tot[o + 1], __dadd_ru(1.0, rel)), ms));
    }
    const double p = P.p;
    const double inv_hi = s_lo > 0.0 ? __drcp_ru(s_lo) : HUGE_VAL;
    const double inv_lo = __drcp_rd(s_hi);
    const double dinv = fmax(0.0, fmax(__dsub_ru(inv_hi, 1.0), __dsub_ru(1.0, inv_lo)));
    const double tv_mu = __fma_ru(tot[12], dinv, __dmul_ru(A[0], inv_hi));
    const double tv_nu = __fma_ru(tot[13], dinv, __dmul_ru(A[1], inv_hi));
    const double scale = (p == 1.0) ? 1.0 : (p == 2.0 ? 2.0 : __dmul_ru(pow(2.0, p - 1.0), 1.0 + 0x1p-49));
    const double dmu = root_p_ru(__dmul_ru(scale, tv_mu), p);
    const double dnu = root_p_ru(__dmul_ru(scale, tv_nu), p);
    const double w_hat_p = __dmul_ru(tot[14], inv_hi);
    PairOut& O = outs[P.out_index];
    O.w_hat_p = w_hat_p;
    O.delta_mu = dmu;
    O.delta_nu = dnu;
    O.ub_primal = __dadd_ru(__dadd_ru(root_p_ru(w_hat_p, p), dmu), dnu);
    O.ipf_residual = tot[4] + tot[10];
    O.sweeps_done = P.sweeps;
}

template <int KK>
__global__ void __launch_bounds__(PKE_THREADS)
primalk_eval_layout_kernel(const PairDev* __restrict__ pairs, const int* __restrict__ pair_ids, int n_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const PairDev& P = pairs[pair_ids[blockIdx.x / n_max]];
    const int k1 = blockIdx.x % n_max, n = P.n, N = P.N, kap = P.kappa;
    if (k1 >= n) return;
    float* tmp = reinterpret_cast<float*>(smem_raw);          // [2][n KK]
    const int t0 = k1 * n * KK, tn = n * KK;
    float* a = reinterpret_cast<float*>(P.a);
    float* b = reinterpret_cast<float*>(P.b);
    for (int t = threadIdx.x; t < tn; t += blockDim.x) {
        tmp[t] = a[t0 + t];
        tmp[tn + t] = b[t0 + t];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < tn; t += blockDim.x) {
        const int tt = t0 + t;
        const int i = blk_pixel(tt / KK, tt - (tt / KK) * KK, n, kap, N);   // in the same rows
        a[i] = tmp[t];
        b[i] = tmp[tn + t];
    }
}

int launch_primalk_eval(const PairDev* pairs_d, PairOut* outs_d, const int* pair_ids, int n_pairs, int kappa,
                        int n_max, cudaStream_t stream) {
    if (n_pairs <= 0) return QWB_OK;
    if (kappa != 2 && kappa != 4 && kappa != 8) return QWB_ERR_UNSUPPORTED;
    const int kk = kappa * kappa;
    const size_t s_kd = sizeof(float) * 2 * (size_t)kk * kk, s_sum = sizeof(float) * (size_t)kk * kk;
    const size_t s_lay = sizeof(float) * 2 * (size_t)n_max * kk;
    if (s_lay > 227 * 1024) return QWB_ERR_UNSUPPORTED;
    const unsigned grid = (unsigned)(n_pairs * n_max);
    auto run = [&](auto kd, auto sum, auto fin, auto lay) -> int {
        QWB_CUDA(cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_kd));
        QWB_CUDA(cudaFuncSetAttribute(lay, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_lay));
        kd<<<grid, PKE_THREADS, s_kd, stream>>>(pairs_d, pair_ids, n_max);
        QWB_LAUNCHED();
        sum<<<grid, PKE_THREADS, s_sum, stream>>>(pairs_d, pair_ids, n_max);
        QWB_LAUNCHED();
        fin<<<n_pairs, 32, 0, stream>>>(pairs_d, outs_d, pair_ids);
        QWB_LAUNCHED();
        lay<<<grid, PKE_THREADS, s_lay, stream>>>(pairs_d, pair_ids, n_max);
        QWB_LAUNCHED();
        return QWB_OK;
    };
    if (kk == 4)
        return run(primalk_eval_kd_kernel<4>, primalk_eval_sum_kernel<4>, primalk_eval_final_kernel<4>,
                   primalk_eval_layout_kernel<4>);
    if (kk == 16)
        return run(primalk_eval_kd_kernel<16>, primalk_eval_sum_kernel<16>, primalk_eval_final_kernel<16>,
                   primalk_eval_layout_kernel<16>);
    return run(primalk_eval_kd_kernel<64>, primalk_eval_sum_kernel<64>, primalk_eval_final_kernel<64>,
               primalk_eval_layout_kernel<64>);
}

// --------------------------------------------------------------------------
// ipf_fine: the fine FP32 IPF sweeps of the primal pass (Sec. 3.4, IPF
// paragraph; Alg. 4), a = mu / (pi-hat b), b = nu / (pi-hat^T a), for large
// 2-D pairs (block side kappa 4 or 8) on a thread-block cluster of C CTAs
// per pair.  CTA `rank` owns the coarse block rows [rank R, (rank+1) R),
// R = ceil(n / C), i.e. the blocks [rank R n, (rank+1) R n) clipped to M
// (whole block rows, so its fine pixels are contiguous rows; the last CTAs
// may own fewer rows or none): it streams
// their pixels, keeps their block sums in its shared memory and reads the
// other CTAs' block sums through distributed shared memory for the coarse
// products r = kappa^-4 pi~ B and s = kappa^-4 pi~^T A.  Each half sweep
// publishes its block sums, arrives at the cluster barrier (release),
// streams the scaled values to memory and prefetches the next half's first
// source values while the barrier completes, then waits (acquire).  The same
// arithmetic as the single-CTA sweeps of primal_kernel, which skips them for
// these pairs (fine_ext): per block one FP32 reciprocal of r and a scaled
// store of every fine value, block sums in FP32.  Every CTA of a cluster runs
// the same number of half sweeps and arrives once per half sweep, so the
// barrier cannot wait on a CTA that has left.
// --------------------------------------------------------------------------
constexpr int IPF_THREADS = 256;                         // the bulk-copy form; the register form: TH

__device__ __forceinline__ void cluster_arrive_release() {
    asm volatile("barrier.cluster.arrive.release;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
    asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory");
}

template <int KAP, int TH>
__global__ void __launch_bounds__(TH)
ipf_fine_kernel(const PairDev* __restrict__ pairs, const int* __restrict__ pair_ids, int C,
                int csr_cap) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int rank = (int)cl.block_rank();
    const PairDev& P = pairs[pair_ids[blockIdx.x / C]];
    const int N = P.N, n = P.n, M = P.M;
    const int Rn = ((n + C - 1) / C) * n;                     // blocks per CTA (the same stride in all)
    const int k0 = min(M, rank * Rn);
    const int Mc = min(M, k0 + Rn) - k0;                      // owned blocks [k0, k0 + Mc)
    float* Aown = reinterpret_cast<float*>(smem_raw);         // block sums of a (owned)
    float* Bown = Aown + Rn;                                  // block sums of b (owned)
    float* v_s = Bown + Rn;                                   // plan values: owned CSR rows
    float* vc_s = v_s + csr_cap;                              //              owned CSC columns
    int* ci_s = reinterpret_cast<int*>(vc_s + csr_cap);
    int* ri_s = ci_s + csr_cap;
    int* rp_s = ri_s + csr_cap;                               // Mc + 1, relative offsets
    int* cp_s = rp_s + Rn + 1;
    const int r_base = P.rowptr[k0], c_base = P.colptr[k0];
    const int r_cnt = P.rowptr[k0 + Mc] - r_base, c_cnt = P.colptr[k0 + Mc] - c_base;
    const bool staged = r_cnt <= csr_cap && c_cnt <= csr_cap;
    const float* vt = reinterpret_cast<const float*>(P.val_t);
    const float* vct = reinterpret_cast<const float*>(P.valc_t);
    if (staged) {
        for (int k = threadIdx.x; k <= Mc; k += blockDim.x) {
            rp_s[k] = P.rowptr[k0 + k] - r_base;
            cp_s[k] = P.colptr[k0 + k] - c_base;
        }
        for (int e = threadIdx.x; e < r_cnt; e += blockDim.x) { ci_s[e] = P.colidx[r_base + e]; v_s[e] = vt[r_base + e]; }
        for (int e = threadIdx.x; e < c_cnt; e += blockDim.x) { ri_s[e] = P.rowidx[c_base + e]; vc_s[e] = vct[c_base + e]; }
    }
    constexpr int KK = KAP * KAP;
    const float kinvK = 1.0f / (float)(KK * KK);              // kappa^-4, exact (a power of two)
    for (int k = threadIdx.x; k < Mc; k += blockDim.x) Bown[k] = (float)KK;   // b = 1
    const float* mu_t = reinterpret_cast<const float*>(P.mu_t);
    const float* nu_t = reinterpret_cast<const float*>(P.nu_t);
    float* a = reinterpret_cast<float*>(P.a);
    float* bb = reinterpret_cast<float*>(P.b);
    constexpr int Q = KAP / 4;                                // float4 per block row
    constexpr int PF = KAP == 4 ? 4 : 1;                      // blocks per chunk and thread
    const int chunk = PF * blockDim.x;
    float4 x[PF][KAP][Q];
    // kappa = 8: when a warp's 32 blocks are all owned and lie in one block
    // row, the warp moves each fine row of them as 64 consecutive float4
    // (lane L holds float4 L and L + 32: half a row of block L / 2 and of
    // block L / 2 + 16), so every load and store instruction covers 512
    // contiguous bytes; each block's scale comes from its owner lane and its
    // sum from the lane pair that holds it.  Other warps keep one block per
    // thread.  The choice depends on the warp's first block only, so the
    // loads, the scaling and the stores of a chunk agree.
    const int lane = threadIdx.x & 31;
    auto row_mode = [&](int kb) {
        if constexpr (KAP != 8) return false;
        const int kw = kb - lane;                              // the warp's first owned block
        if (kw + 31 >= Mc) return false;
        const int kf = k0 + kw;
        return (kf % n) + 31 < n;
    };
    auto load_chunk = [&](const float* src, int kb) {
        if constexpr (KAP == 8) {
            if (row_mode(kb)) {
                const int kf = k0 + kb - lane;
                const int k1 = kf / n, k2 = kf - (kf / n) * n;
#pragma unroll
                for (int t1 = 0; t1 < KAP; ++t1) {
                    const float4* span = reinterpret_cast<const float4*>(src + (size_t)(k1 * KAP + t1) * N + k2 * KAP);
                    x[0][t1][0] = span[lane];
                    x[0][t1][1] = span[lane + 32];
                }
                return;
            }
        }
#pragma unroll
        for (int q = 0; q < PF; ++q) {
            const int kl = kb + q * blockDim.x;
            if (kl < Mc) {
                const int k = k0 + kl;
                const int k1 = k / n, k2 = k - (k / n) * n;
#pragma unroll
                for (int t1 = 0; t1 < KAP; ++t1)
#pragma unroll
                    for (int t2 = 0; t2 < Q; ++t2)
                        x[q][t1][t2] = *reinterpret_cast<const float4*>(src + (size_t)(k1 * KAP + t1) * N +
                                                                         k2 * KAP + 4 * t2);
            }
        }
    };
    if (P.sweeps > 0) load_chunk(mu_t, threadIdx.x);           // first half's first chunk
    cl.sync();                                                  // staging and b = 1 visible
    const int halves = 2 * P.sweeps;
    for (int h = 0; h < halves; ++h) {
        const int half = h & 1;
        const float* src = half == 0 ? mu_t : nu_t;
        float* dst = half == 0 ? a : bb;
        float* mine = half == 0 ? Aown : Bown;
        const float* other = half == 0 ? Bown : Aown;
        bool arrived = false;
        for (int kb = threadIdx.x; kb < Mc; kb += chunk) {
            if (kb != (int)threadIdx.x) load_chunk(src, kb);   // later chunks (the first is prefetched)
            float inv[PF];
#pragma unroll
            for (int q = 0; q < PF; ++q) {
                const int kl = kb + q * blockDim.x;
                inv[q] = 0.0f;
                if (kl < Mc) {
                    float r = 0.0f;
                    const int* ptr = staged ? (half == 0 ? rp_s : cp_s) : (half == 0 ? P.rowptr : P.colptr);
                    const int* idx = staged ? (half == 0 ? ci_s : ri_s) : (half == 0 ? P.colidx : P.rowidx);
                    const float* val = staged ? (half == 0 ? v_s : vc_s) : (half == 0 ? vt : vct);
                    const int row = staged ? kl : k0 + kl;
                    for (int e = ptr[row]; e < ptr[row + 1]; ++e) {
                        const int l = idx[e], owner = l / Rn;
                        const float* peer = cl.map_shared_rank(other, owner);
                        r += val[e] * peer[l - owner * Rn];
                    }
                    r *= kinvK;
                    inv[q] = r > 0.0f ? 1.0f / r : 0.0f;
                }
            }
            const bool rows = row_mode(kb);
            if (rows) {
                if constexpr (KAP == 8) {
                    const int kw = kb - lane;
#pragma unroll
                    for (int hq = 0; hq < 2; ++hq) {             // half rows of block lane / 2 + 16 hq
                        const float sc = __shfl_sync(0xffffffffu, inv[0], lane / 2 + 16 * hq);
                        float s = 0.0f;
#pragma unroll
                        for (int t1 = 0; t1 < KAP; ++t1) {
                            float4& v = x[0][t1][hq];
                            v.x *= sc; v.y *= sc; v.z *= sc; v.w *= sc;
                            s += (v.x + v.y) + (v.z + v.w);
                        }
                        s += __shfl_xor_sync(0xffffffffu, s, 1);
                        if (!(lane & 1)) mine[kw + lane / 2 + 16 * hq] = s;
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < PF; ++q) {
                    const int kl = kb + q * blockDim.x;
                    if (kl < Mc) {
                        float s = 0.0f;
#pragma unroll
                        for (int t1 = 0; t1 < KAP; ++t1)
#pragma unroll
                            for (int t2 = 0; t2 < Q; ++t2) {
                                float4& v = x[q][t1][t2];
                                v.x *= inv[q]; v.y *= inv[q]; v.z *= inv[q]; v.w *= inv[q];
                                s += (v.x + v.y) + (v.z + v.w);
                            }
                        mine[kl] = s;
                    }
                }
            }
            if (kb + chunk >= Mc) { cluster_arrive_release(); arrived = true; }   // sums published
            if (rows) {
                if constexpr (KAP == 8) {
                    const int kf = k0 + kb - lane;
                    const int k1 = kf / n, k2 = kf - (kf / n) * n;
#pragma unroll
                    for (int t1 = 0; t1 < KAP; ++t1) {
                        float4* span = reinterpret_cast<float4*>(dst + (size_t)(k1 * KAP + t1) * N + k2 * KAP);
                        span[lane] = x[0][t1][0];
                        span[lane + 32] = x[0][t1][1];
                    }
                }
                continue;
            }
#pragma unroll
            for (int q = 0; q < PF; ++q) {
                const int kl = kb + q * blockDim.x;
                if (kl < Mc) {
                    const int k = k0 + kl;
                    const int k1 = k / n, k2 = k - (k / n) * n;
#pragma unroll
                    for (int t1 = 0; t1 < KAP; ++t1)
#pragma unroll
                        for (int t2 = 0; t2 < Q; ++t2)
                            *reinterpret_cast<float4*>(dst + (size_t)(k1 * KAP + t1) * N + k2 * KAP + 4 * t2) =
                                x[q][t1][t2];
                }
            }
        }
        if (!arrived) cluster_arrive_release();                 // threads without blocks
        if (h + 1 < halves) load_chunk(half == 0 ? nu_t : mu_t, threadIdx.x);   // next half, first chunk
        cluster_wait_acquire();
    }
}

int launch_ipf_fine(const PairDev* pairs_d, const int* pair_ids, int n_pairs, int kappa, int C,
                    int M_max, int nnz_max, cudaStream_t stream, int threads) {
    if (n_pairs <= 0) return QWB_OK;
    if (C < 1 || C > 16 || (kappa != 4 && kappa != 8) || (threads != 256 && threads != 512))
        return QWB_ERR_UNSUPPORTED;
    int n_max = 1;                                            // square grids: M = n^2
    while ((n_max + 1) * (n_max + 1) <= M_max) ++n_max;
    const int Mc = ((n_max + C - 1) / C) * n_max;             // blocks per CTA at most
    // staged plan rows and columns of one CTA: a basic plan has at most 2M - 1
    // entries, on average 2 per owned block; room for twice that (a CTA whose
    // blocks hold more reads its part of the plan from global memory)
    int csr_cap = std::max(nnz_max, 4 * Mc);
    size_t smem = sizeof(float) * 2 * (size_t)Mc + 2 * (sizeof(float) + sizeof(int)) * (size_t)csr_cap +
                  2 * sizeof(int) * (size_t)(Mc + 1);
    if (smem > 100 * 1024) {
        smem = sizeof(float) * 2 * (size_t)Mc + 2 * sizeof(int) * (size_t)(Mc + 1);
        csr_cap = 0;
    }
    auto kern = threads == 512 ? (kappa == 4 ? ipf_fine_kernel<4, 512> : ipf_fine_kernel<8, 512>)
                               : (kappa == 4 ? ipf_fine_kernel<4, 256> : ipf_fine_kernel<8, 256>);
    QWB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (C > 8) QWB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_pairs * C));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    QWB_CUDA(cudaLaunchKernelEx(&cfg, kern, pairs_d, pair_ids, C, csr_cap));
    QWB_LAUNCHED();
    return QWB_OK;
}

// --------------------------------------------------------------------------
// ipf_stream: the same fine FP32 IPF sweeps as ipf_fine_kernel (same cluster
// ownership, block sums through distributed shared memory, one cluster
// barrier per half sweep), with the source values staged by bulk copies.
// A CTA owns nbr = n / C whole block rows, i.e. a contiguous range of pixel
// rows.  Each half sweep is cut into chunks of rps block rows (about 16 KB);
// one thread keeps a ring of PK_STAGES chunks in flight with
// cp.async.bulk (completion counted in bytes on one mbarrier per stage), and
// keeps issuing across half-sweep boundaries, since the sources mu, nu do not
// depend on the sweeps.  Per half sweep the CTA first forms
// r = kappa^-4 pi~ B for its blocks (1 / r in shared memory), then per chunk:
// wait for the stage, scale its values row-major (float4 from shared memory,
// coalesced float4 stores), write per-row block partial sums, barrier,
// re-issue the stage, and reduce the partials over the block's kappa rows in
// a fixed order (the sums match ipf_fine_kernel's association only up to
// rounding; both are FP32 sweeps outside the certificate).  Every wait on an
// mbarrier is bounded: on time-out the CTA sets *err, stops issuing copies
// and processing, and still takes part in every barrier, so no CTA of the
// cluster is left waiting; before returning it waits, bounded again, for the
// copies it issued.
// --------------------------------------------------------------------------
constexpr int PK_STAGES = 4;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(bar), "r"(phase) : "memory");
    return done != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait: false once timeout_ns nanoseconds of the global timer have
// passed without the phase completing (each poll may suspend the thread)
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase, unsigned long long timeout_ns) {
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, phase)) return true;
        if (global_ns() - t0 > timeout_ns) return false;
    }
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

template <int KAP>
__global__ void __launch_bounds__(IPF_THREADS)
ipf_stream_kernel(const PairDev* __restrict__ pairs, const int* __restrict__ pair_ids, int C, int rps,
                  int stage_bytes, int* __restrict__ err, unsigned long long timeout_ns, int skip_chunk) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int rank = (int)cl.block_rank();
    const PairDev& P = pairs[pair_ids[blockIdx.x / C]];
    const int N = P.N, n = P.n;
    const int nbr = n / C, kr0 = rank * nbr;                  // owned block rows
    const int Mc = nbr * n, k0 = kr0 * n;                     // owned blocks [k0, k0 + Mc)
    const int nch = nbr / rps;                                // chunks per half sweep
    const int R = rps * KAP;                                  // pixel rows per chunk
    const int F4 = R * N / 4;                                 // float4 per chunk
    // [stages | mbarriers | Aown, Bown, inv (Mc each) | partial sums (2 x R x n)]
    unsigned char* stages = smem_raw;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)PK_STAGES * stage_bytes);
    float* Aown = reinterpret_cast<float*>(bars + PK_STAGES);
    float* Bown = Aown + Mc;
    float* inv_s = Bown + Mc;
    float* psum = inv_s + Mc;
    constexpr int KK = KAP * KAP;
    const float kinvK = 1.0f / (float)(KK * KK);              // kappa^-4, exact (a power of two)
    const int halves = 2 * P.sweeps;
    const int total = halves * nch;                           // chunks over the whole launch
    const float* mu_t = reinterpret_cast<const float*>(P.mu_t);
    const float* nu_t = reinterpret_cast<const float*>(P.nu_t);
    float* a = reinterpret_cast<float*>(P.a);
    float* bb = reinterpret_cast<float*>(P.b);
    const size_t row0 = (size_t)kr0 * KAP * N;                // first owned pixel row, as a float offset
    bool bad = false;                                         // a wait of this thread timed out
    int issued = 0, waited = 0;                               // thread 0: chunks issued / waited for
    auto issue = [&](int gi) {                                // thread 0: chunk gi into stage gi % PK_STAGES
        if (gi >= total) return;
        issued = gi + 1;
        if (gi == skip_chunk) return;                         // host-requested fault: never issued
        const int h = gi / nch, c = gi - (gi / nch) * nch;
        const float* src = ((h & 1) == 0 ? mu_t : nu_t) + row0 + (size_t)c * R * N;
        const int s = gi % PK_STAGES;
        const uint32_t bar = smem_addr(bars + s);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_expect_tx(bar, (uint32_t)stage_bytes);
        bulk_load(smem_addr(stages + (size_t)s * stage_bytes), src, (uint32_t)stage_bytes, bar);
    };
    if (threadIdx.x == 0) {
        for (int s = 0; s < PK_STAGES; ++s) mbar_init(smem_addr(bars + s), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int k = threadIdx.x; k < Mc; k += blockDim.x) Bown[k] = (float)KK;   // b = 1
    __syncthreads();
    if (threadIdx.x == 0)
        for (int gi = 0; gi < PK_STAGES; ++gi) issue(gi);
    cl.sync();                                                // b = 1 visible to the cluster
    const int lane = threadIdx.x & 31;
    const int n_f = (F4 + blockDim.x - 1) / blockDim.x;       // the same trip count for every thread
    for (int h = 0; h < halves; ++h) {
        const int half = h & 1;
        float* dst = half == 0 ? a : bb;
        float* mine = half == 0 ? Aown : Bown;
        const float* other = half == 0 ? Bown : Aown;
        // 1 / r for the owned blocks (coarse product over the plan row / column;
        // staging the plan in shared memory measured slower: fewer resident CTAs)
        const int* ptr = half == 0 ? P.rowptr : P.colptr;
        const int* idx = half == 0 ? P.colidx : P.rowidx;
        const float* val = reinterpret_cast<const float*>(half == 0 ? P.val_t : P.valc_t);
        for (int kl = threadIdx.x; kl < Mc; kl += blockDim.x) {
            float r = 0.0f;
            for (int e = ptr[k0 + kl]; e < ptr[k0 + kl + 1]; ++e) {
                const int l = idx[e], owner = l / Mc;
                const float* peer = cl.map_shared_rank(other, owner);
                r += val[e] * peer[l - owner * Mc];
            }
            r *= kinvK;
            inv_s[kl] = r > 0.0f ? 1.0f / r : 0.0f;
        }
        __syncthreads();
        for (int c = 0; c < nch; ++c) {
            const int gi = h * nch + c, s = gi % PK_STAGES;
            const uint32_t phase = (uint32_t)((gi / PK_STAGES) & 1);
            if (!bad && !mbar_wait_bounded(smem_addr(bars + s), phase, timeout_ns)) {
                bad = true;
                atomicOr(err, 1);
            }
            if (!bad) waited = gi + 1;
            const float4* st4 = reinterpret_cast<const float4*>(stages + (size_t)s * stage_bytes);
            float4* d4 = reinterpret_cast<float4*>(dst + row0 + (size_t)c * R * N);
            float* ps = psum + (c & 1) * R * n;
            for (int j = 0; j < n_f; ++j) {
                const int f = threadIdx.x + j * blockDim.x;
                const bool ok = f < F4 && !bad;
                float part = 0.0f;
                int pr = 0, kc = 0;
                if (ok) {
                    pr = (4 * f) / N;
                    const int col = 4 * f - pr * N;
                    kc = col / KAP;
                    const float iv = inv_s[(c * rps + pr / KAP) * n + kc];
                    float4 v = st4[f];
                    v.x *= iv; v.y *= iv; v.z *= iv; v.w *= iv;
                    d4[f] = v;
                    part = (v.x + v.y) + (v.z + v.w);
                }
                if (KAP == 8) part += __shfl_xor_sync(0xffffffffu, part, 1);   // the row's two float4 of the block
                if (ok && (KAP == 4 || (lane & 1) == 0)) ps[pr * n + kc] = part;
            }
            __syncthreads();                                  // stage read, partial sums written
            if (threadIdx.x == 0 && !bad) issue(gi + PK_STAGES);
            for (int q = threadIdx.x; q < rps * n; q += blockDim.x) {
                const int lbr = q / n, kc = q - (q / n) * n;
                float sum = 0.0f;
#pragma unroll
                for (int t1 = 0; t1 < KAP; ++t1) sum += ps[(lbr * KAP + t1) * n + kc];
                mine[(c * rps + lbr) * n + kc] = sum;
            }
        }
        cluster_arrive_release();                             // this half's block sums published
        cluster_wait_acquire();
    }
    // copies issued but not waited for (none when every wait succeeded; at
    // most PK_STAGES otherwise): wait, bounded, before the CTA leaves
    if (threadIdx.x == 0)
        for (int gi = waited; gi < issued; ++gi)
            if (gi != skip_chunk)
                (void)mbar_wait_bounded(smem_addr(bars + gi % PK_STAGES), (uint32_t)((gi / PK_STAGES) & 1),
                                        timeout_ns);
}

// chunk rows (block rows per stage) for a pair of the group: the largest
// divisor of n / C with at most 16 KB per chunk (at least one block row)
static int ipf_stream_rps(int n, int C, int kappa, int N) {
    const int nbr = n / C;
    int best = 1;
    for (int r = 1; r <= nbr; ++r)
        if (nbr % r == 0 && (size_t)r * kappa * N * sizeof(float) <= 16384) best = r;
    return best;
}

int launch_ipf_stream(const PairDev* pairs_d, const int* pair_ids, int n_pairs, int kappa, int C, int n,
                      int N, int* err, unsigned long long timeout_ns, int skip_chunk, cudaStream_t stream) {
    if (n_pairs <= 0) return QWB_OK;
    if (C < 1 || C > 16 || (kappa != 4 && kappa != 8) || n % C != 0 || N % 4 != 0) return QWB_ERR_UNSUPPORTED;
    const int rps = ipf_stream_rps(n, C, kappa, N);
    const int stage_bytes = rps * kappa * N * (int)sizeof(float);
    const int Mc = (n / C) * n;
    const size_t smem = (size_t)PK_STAGES * stage_bytes + PK_STAGES * sizeof(uint64_t) +
                        3 * sizeof(float) * (size_t)Mc + 2 * sizeof(float) * (size_t)rps * kappa * n;
    if (smem > 220 * 1024) return QWB_ERR_UNSUPPORTED;
    auto kern = kappa == 4 ? ipf_stream_kernel<4> : ipf_stream_kernel<8>;
    QWB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (C > 8) QWB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_pairs * C));
    cfg.blockDim = dim3(IPF_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    QWB_CUDA(cudaLaunchKernelEx(&cfg, kern, pairs_d, pair_ids, C, rps, stage_bytes, err, timeout_ns, skip_chunk));
    QWB_LAUNCHED();
    return QWB_OK;
}

// --------------------------------------------------------------------------
// centre: s = <f~, mu~> so that the upscaled potential is f~ - s (the lower
// bound is invariant to such shifts because both measures have mass 1).
// --------------------------------------------------------------------------
__global__ void centre_kernel(const PairDev* __restrict__ pairs, PairOut* __restrict__ outs,
                              const int* __restrict__ pair_ids, int side) {
    __shared__ double red[33];
    const PairDev& P = pairs[pair_ids[blockIdx.x]];
    // side 0: <f~, mu~>; side 1 (upscaling from g~): <g~, nu~>
    const double* pc = side ? P.g_coarse : P.f_coarse;
    const double* wc = side ? P.nu_c : P.mu_c;
    double s = 0.0;
    for (int k = threadIdx.x; k < P.M; k += blockDim.x) s += pc[k] * wc[k];
    s = block_reduce_rn(s, red);
    if (threadIdx.x == 0) outs[P.out_index].centre_shift = s;
}

int launch_centre(const PairDev* pairs_d, PairOut* outs_d, const int* pair_ids, int n_pairs,
                  cudaStream_t stream, int side) {
    if (n_pairs <= 0) return QWB_OK;
    centre_kernel<<<n_pairs, 256, 0, stream>>>(pairs_d, outs_d, pair_ids, side);
    QWB_LAUNCHED();
    return QWB_OK;
}

// --------------------------------------------------------------------------
// upsample: f-hat(x) = R_{f~ - s}(x), bilinear in block-centre coordinates
// t = (x - (kappa-1)/2) / kappa with linear extrapolation at the border
// (Sec. 3.5; Alg. 5).  Also resets the c-transform outputs to +inf when they
// are combined with atomics.
// --------------------------------------------------------------------------
template <typename T>
__global__ void upsample_kernel(const PairDev* __restrict__ pairs, const PairOut* __restrict__ outs,
                                const PixItem* __restrict__ items, int side) {
    const PixItem I = items[blockIdx.x];
    const PairDev& P = pairs[I.pair];
    const int i = I.start + threadIdx.x;
    const int N = P.N, n = P.n, kap = P.kappa;
    if (i >= P.m) return;
    const double s = outs[P.out_index].centre_shift;
    const double* fc = side ? P.g_coarse : P.f_coarse;   // the coarse potential upscaled
    const int r = P.d == 3 ? i / (N * N) : i / N, c = P.d == 3 ? (i / N) % N : i % N;
    double v;
    if (n == 1) {
        v = fc[0] - s;
    } else if (P.d == 3) {
        // trilinear: interpolate along the first axis, then the second, then
        // the third (the tensor-product rule, per axis as in two dimensions)
        const int z = i % N;
        const int den = 2 * kap;
        const double inv = 1.0 / den;
        int k0[3];
        double w[3];
        const int x[3] = {r, c, z};
        for (int a = 0; a < 3; ++a) {
            const int num = 2 * x[a] - kap + 1;
            const int fl = num >= 0 ? num / den : -((-num + den - 1) / den);
            k0[a] = min(max(fl, 0), n - 2);
            w[a] = (double)(num - den * k0[a]) * inv;
        }
        double h[2];
        for (int e3 = 0; e3 < 2; ++e3) {
            double g2[2];
            for (int e2 = 0; e2 < 2; ++e2) {
                const int b = ((k0[0]) * n + k0[1] + e2) * n + k0[2] + e3;
                g2[e2] = (1.0 - w[0]) * (fc[b] - s) + w[0] * (fc[b + n * n] - s);
            }
            h[e3] = (1.0 - w[1]) * g2[0] + w[1] * g2[1];
        }
        v = (1.0 - w[2]) * h[0] + w[2] * h[1];
    } else {
        // t = (x - (kappa-1)/2) / kappa = (2x - kappa + 1) / (2 kappa): the cell
        // index by integer floor division, the weight from the integer
        // remainder (one reciprocal per thread instead of two divisions)
        const int den = 2 * kap, nr = 2 * r - kap + 1, nc = 2 * c - kap + 1;
        const int flr = nr >= 0 ? nr / den : -((-nr + den - 1) / den);
        const int flc = nc >= 0 ? nc / den : -((-nc + den - 1) / den);
        const int r0 = min(max(flr, 0), n - 2), c0 = min(max(flc, 0), n - 2);
        const int qr = nr - den * r0, qc = nc - den * c0;          // weights qr / den, qc / den
        double wr, wc, wr1, wc1;                                   // and 1 - each
        if (!(kap & (kap - 1))) {
            // den a power of two: q / den and (den - q) / den are exact in
            // FP32 (|q| < 2^24) and widen exactly, the same values as the
            // FP64 expressions below, without the FP64 pipe
            const float id = __frcp_rn((float)den);
            wr = widen_f32((float)qr * id); wc = widen_f32((float)qc * id);
            wr1 = widen_f32((float)(den - qr) * id); wc1 = widen_f32((float)(den - qc) * id);
        } else {
            const double inv = 1.0 / den;
            wr = (double)qr * inv; wc = (double)qc * inv;
            wr1 = 1.0 - wr; wc1 = 1.0 - wc;
        }
        const double f00 = fc[r0 * n + c0] - s, f01 = fc[r0 * n + c0 + 1] - s;
        const double f10 = fc[(r0 + 1) * n + c0] - s, f11 = fc[(r0 + 1) * n + c0 + 1] - s;
        const double top = wc1 * f00 + wc * f01;
        const double bot = wc1 * f10 + wc * f11;
        v = wr1 * top + wr * bot;
    }
    reinterpret_cast<T*>(P.fhat)[i] = from_double_rn<T>(v);
    reinterpret_cast<T*>(P.g)[i] = pos_inf<T>();     // c-transform outputs start at +inf
    reinterpret_cast<T*>(P.f)[i] = pos_inf<T>();
}

// --------------------------------------------------------------------------
// verify: the certificate check of a dual pass.  The lower bound rests on the
// admissibility of the pair (f, g): f_i + g_j <= c_ij for every pair of fine
// points (the dual constraint of Sec. 2.1, which the c-transforms of Sec. 3.5
// restore).  One thread per output point j; the input rows of f are staged
// through shared memory.  Each sum is rounded upward and compared with a
// lower bracket of the cost (the exact integer for p = 2, the cost table's
// lower bracket otherwise), so a pass proves admissibility; a failure sets
// the pair's flag.  2-D pairs only (volumes are skipped).
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
verify_kernel(const PairDev* __restrict__ pairs, PairOut* __restrict__ outs, const PixItem* __restrict__ items,
              T shift) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* frow = reinterpret_cast<T*>(smem_raw);                 // one row of f (N values)
    const PixItem I = items[blockIdx.x];
    const PairDev& P = pairs[I.pair];
    const int N = P.N, m = P.m;
    if (P.d != 2 || (size_t)N * sizeof(T) > 48 * 1024) return;   // the whole CTA leaves
    const int j = I.start + threadIdx.x;
    const bool valid = j < m;
    const T* f = reinterpret_cast<const T*>(P.f);
    const T gj = valid ? reinterpret_cast<const T*>(P.g)[j] : T(0);
    const int j1 = valid ? j / N : 0, j2 = valid ? j - j1 * N : 0;
    const bool p2 = P.p == 2.0 && N <= 2896;                  // squared offsets exact in FP32
    const T* tab = reinterpret_cast<const T*>(P.ctab_lo);
    int bad = 0;
    for (int i1 = 0; i1 < N; ++i1) {
        __syncthreads();
        for (int q = threadIdx.x; q < N; q += blockDim.x) frow[q] = f[(size_t)i1 * N + q];
        __syncthreads();
        if (!valid) continue;
        const int di1 = abs(i1 - j1);
        const T a = (T)(di1 * di1);
        const T* trow = tab + (size_t)di1 * N;
        for (int i2 = 0; i2 < N; ++i2) {
            const int d2 = i2 - j2;
            const T c = p2 ? a + (T)(d2 * d2) : trow[abs(d2)];
            bad |= add_ru(frow[i2], gj) > c - shift;
        }
    }
    if (bad) atomicOr(&outs[P.out_index].verify_bad, 1);
}

int launch_verify(const PairDev* pairs_d, PairOut* outs_d, const PixItem* items, int n_items, bool f64,
                  double shift, cudaStream_t stream) {
    if (n_items <= 0) return QWB_OK;
    // shared memory: one row of f for the largest side the items can have
    // (at most the 48 KB default: N <= 6144 in FP64)
    const size_t smem = 48 * 1024;
    if (f64) verify_kernel<double><<<n_items, 256, smem, stream>>>(pairs_d, outs_d, items, shift);
    else verify_kernel<float><<<n_items, 256, smem, stream>>>(pairs_d, outs_d, items, (float)shift);
    QWB_LAUNCHED();
    return QWB_OK;
}

int launch_upsample(const PairDev* pairs_d, PairOut* outs_d, const PixItem* items, int n_items,
                    bool f64, cudaStream_t stream, int side) {
    if (n_items <= 0) return QWB_OK;
    if (f64) upsample_kernel<double><<<n_items, 256, 0, stream>>>(pairs_d, outs_d, items, side);
    else upsample_kernel<float><<<n_items, 256, 0, stream>>>(pairs_d, outs_d, items, side);
    QWB_LAUNCHED();
    return QWB_OK;
}

// --------------------------------------------------------------------------
// Separable c-transform for p = 2 (squared Euclidean cost on the grid):
//   min over (i1, i2) of (i1-j1)^2 + (i2-j2)^2 - h(i1,i2)
//     = min over i1 of (i1-j1)^2 + t(i1, j2),   t(i1, j2) = min over i2 of (i2-j2)^2 - h(i1,i2),
// two one-dimensional transforms of N^3 candidate pairs each instead of N^4.
// One launch is one stage over lines of N values:
//   out[j * N + r] = sign * min_i fl_down((i - j)^2 - in[r * N + i])
// stage 1: in = h, sign = -1, out = the scratch (holds -t, transposed);
// stage 2: in = the scratch, sign = +1, out = the result (transposed back).
// Every candidate is rounded toward -inf and minima are exact, so t is at
// most the exact row minimum and the result at most
// (i1-j1)^2 + (i2-j2)^2 - h(i1,i2) for every input: the output is a
// certified c-transform.  Thread t of a line owns SEP_R consecutive outputs
// and walks the inputs in chunks of SEP_TC, with the SEP_R + SEP_TC - 1
// distinct squared offsets of a chunk held in registers (the same register
// blocking as the two-dimensional kernel).  Lines are padded to a multiple of
// SEP_R with -inf inputs (candidates +inf); outputs are staged in shared
// memory and written transposed in contiguous runs.
// --------------------------------------------------------------------------
constexpr int SEP_R = 8, SEP_TC = 8, SEP_THREADS = 256;

int sep_lines_per_cta(int N) {
    const int Lp = (N + SEP_R - 1) / SEP_R * SEP_R;
    return std::max(1, SEP_THREADS / (Lp / SEP_R));
}

template <typename T>
__global__ void __launch_bounds__(SEP_THREADS)
sep_kernel(const PairDev* __restrict__ pairs, const SepItem* __restrict__ items, int n_items,
           int phase, int stage) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NQ = SEP_R + SEP_TC - 1;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const SepItem I = items[it];
        const PairDev& P = pairs[I.pair];
        if (stage >= P.d) continue;                   // fewer axes than this stage
        const int N = P.N, L = P.rows;                // L lines of N points
        const int Lp = (N + SEP_R - 1) / SEP_R * SEP_R;
        const int tpl = Lp / SEP_R;
        const int last = P.d - 1;
        const T* in = reinterpret_cast<const T*>(stage == 0 ? (phase == 0 ? P.fhat : P.g)
                                                             : (stage == 1 ? P.tsep : P.tsep2));
        T* out = reinterpret_cast<T*>(stage == last ? (phase == 0 ? P.g : P.f)
                                                    : (stage == 0 ? P.tsep : P.tsep2));
        T* hs = reinterpret_cast<T*>(smem_raw);                 // [lines][Lp]
        T* os = hs + I.lines * Lp;                              // [lines][Lp + 1]
        for (int k = threadIdx.x; k < I.lines * Lp; k += blockDim.x) {
            const int r = k / Lp, i = k - r * Lp;
            hs[k] = i < N ? in[(size_t)(I.line0 + r) * N + i] : -pos_inf<T>();
        }
        __syncthreads();
        const int line = threadIdx.x / tpl;
        if (line < I.lines) {
            const int j0 = (threadIdx.x - line * tpl) * SEP_R;
            T mins[SEP_R];
#pragma unroll
            for (int r = 0; r < SEP_R; ++r) mins[r] = pos_inf<T>();
            const T* hrow = hs + line * Lp;
            for (int c0 = 0; c0 < Lp; c0 += SEP_TC) {
                T q[NQ];
#pragma unroll
                for (int e = 0; e < NQ; ++e) {
                    const T d = (T)(c0 - j0 + e - (SEP_R - 1));
                    q[e] = d * d;                                // exact integers
                }
                T fv[SEP_TC];
#pragma unroll
                for (int s = 0; s < SEP_TC; ++s) fv[s] = hrow[c0 + s];
#pragma unroll
                for (int s = 0; s < SEP_TC; s += 2)
#pragma unroll
                    for (int r = 0; r < SEP_R; ++r)
                        mins[r] = min3(mins[r], sub_rd(q[s - r + SEP_R - 1], fv[s]),
                                       sub_rd(q[s + 1 - r + SEP_R - 1], fv[s + 1]));
            }
            const T sign = stage == last ? T(1) : T(-1);
#pragma unroll
            for (int r = 0; r < SEP_R; ++r) os[line * (Lp + 1) + j0 + r] = sign * mins[r];
        }
        __syncthreads();
        for (int k = threadIdx.x; k < I.lines * N; k += blockDim.x) {
            const int j = k / I.lines, r = k - j * I.lines;
            out[(size_t)j * L + I.line0 + r] = os[r * (Lp + 1) + j];
        }
        __syncthreads();
    }
}

int launch_sep(const PairDev* pairs_d, const SepItem* items, int n_items, int phase, int stage,
               int N_max, bool f64, int grid_cap, cudaStream_t stream) {
    if (n_items <= 0) return QWB_OK;
    const size_t tsz = f64 ? 8 : 4;
    (void)N_max;
    // per item: lines * Lp <= SEP_THREADS * SEP_R inputs, as many outputs plus
    // one pad per line (at most SEP_THREADS lines)
    const size_t smem = tsz * ((size_t)SEP_THREADS * SEP_R * 2 + SEP_THREADS);
    auto run = [&](auto kern) -> int {
        QWB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int grid = n_items;
        if (grid_cap > 0) {
            int occ = 1;
            QWB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, SEP_THREADS, smem));
            grid = std::min(n_items, grid_cap * std::max(1, occ));
        }
        kern<<<grid, SEP_THREADS, smem, stream>>>(pairs_d, items, n_items, phase, stage);
        QWB_LAUNCHED();
        return QWB_OK;
    };
    return f64 ? run(sep_kernel<double>) : run(sep_kernel<float>);
}

// --------------------------------------------------------------------------
// lbsum: lb_p = <f, mu> + <g, nu> summed with FP64 round-down fused
// multiply-adds, so lb_p <= the real dual objective of the stored (f, g)
// (Sec. 3.5, eq. upscaling LB); LB = max(lb_p, 0)^(1/p) rounded down.
// --------------------------------------------------------------------------
template <typename T>
__global__ void lbsum_kernel(const PairDev* __restrict__ pairs, PairOut* __restrict__ outs,
                             const int* __restrict__ pair_ids, int side) {
    __shared__ double red[33];
    const PairDev& P = pairs[pair_ids[blockIdx.x]];
    const int m = P.m;
    // side 0: the transforms ran f-hat -> g -> f.  Side 1 (upscaling from
    // g~): they ran g-hat -> f -> g, so the buffer named g holds the
    // potential on mu's side and the buffer named f the one on nu's side.
    const T* fm = reinterpret_cast<const T*>(side ? P.g : P.f);
    const T* gn = reinterpret_cast<const T*>(side ? P.f : P.g);
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        s = __fma_rd((double)fm[i], P.mu[i], s);
        s = __fma_rd((double)gn[i], P.nu[i], s);
    }
    s = block_reduce_rd(s, red);
    PairOut& O = outs[P.out_index];
    // the larger of the two certified bounds is kept, with its potentials
    const bool keep = side == 0 || s > O.lb_p;
    if (keep && (P.f_out || P.g_out)) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            if (P.f_out) P.f_out[i] = (double)fm[i];
            if (P.g_out) P.g_out[i] = (double)gn[i];
        }
    }
    if (keep && threadIdx.x == 0) {
        O.lb_p = s;
        O.lb = root_p_rd(fmax(s, 0.0), P.p);
    }
}

int launch_lbsum(const PairDev* pairs_d, PairOut* outs_d, const int* pair_ids, int n_pairs,
                 bool f64, cudaStream_t stream, int side) {
    if (n_pairs <= 0) return QWB_OK;
    if (f64) lbsum_kernel<double><<<n_pairs, 1024, 0, stream>>>(pairs_d, outs_d, pair_ids, side);
    else lbsum_kernel<float><<<n_pairs, 1024, 0, stream>>>(pairs_d, outs_d, pair_ids, side);
    QWB_LAUNCHED();
    return QWB_OK;
}

// --------------------------------------------------------------------------
// adjoint: grad_i = (1/p) lb_p^(1/p - 1) (f_i - <f, mu>)
// --------------------------------------------------------------------------
__global__ void dot_kernel(const double* __restrict__ f, const double* __restrict__ mu, int m,
                           double* out) {
    __shared__ double red[33];
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s += f[i] * mu[i];
    s = block_reduce_rn(s, red);
    if (threadIdx.x == 0) *out = s;
}
__global__ void adjoint_kernel(const double* __restrict__ f, const double* __restrict__ fmu,
                               int m, double scale, double* __restrict__ grad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) grad[i] = scale * (f[i] - *fmu);
}

int launch_adjoint(int N, double p, const double* f, const double* mu, double lb_p, double* grad,
                   double* scratch, cudaStream_t stream) {
    const int m = N * N;
    dot_kernel<<<1, 1024, 0, stream>>>(f, mu, m, scratch);
    QWB_LAUNCHED();
    const double scale = lb_p > 0.0 ? (1.0 / p) * pow(lb_p, 1.0 / p - 1.0) : 0.0;
    adjoint_kernel<<<(m + 255) / 256, 256, 0, stream>>>(f, scratch, m, scale, grad);
    QWB_LAUNCHED();
    return QWB_OK;
}

// --------------------------------------------------------------------------
// Standalone c-transform of a caller potential (FP64 in and out).
// --------------------------------------------------------------------------
template <typename T>
__global__ void to_work_ru(const double* __restrict__ h, T* __restrict__ w, T* __restrict__ o,
                           int m, int init_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    w[i] = from_double_ru<T>(h[i]);
    if (init_out) o[i] = pos_inf<T>();
}
template <typename T>
__global__ void from_work(const T* __restrict__ o, double* __restrict__ out, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) out[i] = (double)o[i];
}

int launch_to_work(const double* h, void* work_in, void* work_out, int m, bool f64,
                   cudaStream_t stream) {
    const int bl = (m + 255) / 256;
    if (f64) to_work_ru<double><<<bl, 256, 0, stream>>>(h, (double*)work_in, (double*)work_out, m, 1);
    else to_work_ru<float><<<bl, 256, 0, stream>>>(h, (float*)work_in, (float*)work_out, m, 1);
    QWB_LAUNCHED();
    return QWB_OK;
}

int launch_from_work(const void* work, double* out, int m, bool f64, cudaStream_t stream) {
    const int bl = (m + 255) / 256;
    if (f64) from_work<double><<<bl, 256, 0, stream>>>((const double*)work, out, m);
    else from_work<float><<<bl, 256, 0, stream>>>((const float*)work, out, m);
    QWB_LAUNCHED();
    return QWB_OK;
}

}  // namespace qwb
