// ctransform.cu -- the lazy min-plus c-transform (Sec. 4, eq. lazy
// c-transform; Alg. 5), the dominant pass of the dual lower bound.
//
// Kept apart from the other passes so that its many compiled launch shapes
// build in parallel with them and so that its source identifies the kernel
// whose counters the DRAM-traffic record refers to.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace qwb {

// --------------------------------------------------------------------------
// ctransform: out_j = min_i fl_down(c_ij - h_i)   (Sec. 4, eq. lazy c-transform)
//
// Work item = (pair, a contiguous range of threads*R outputs, a range of input
// rows).  The input rows are staged in shared memory.  Thread t owns R
// consecutive outputs j = (j1, j2 .. j2+R-1) of one grid row and walks the
// inputs in chunks of TC columns.  For a chunk starting at column c0 and an
// input row i1, the R*TC costs take only R+TC-1 distinct values
//   q_e = rho((i1 - j1, c0 - j2 + e))^p,  e = s - r in [-(R-1), TC-1],
// so each (input, output) pair costs one subtraction rounded toward -inf and
// one min.  For p = 2 the costs are exact integers built from
// (i1-j1)^2 + (c0-j2+e)^2 (the column part is computed once per chunk);
// other p read them from the round-down cost table.  Because every candidate
// is rounded down and the min is exact, h_i + out_j <= c_ij holds exactly.
// Items that cover only part of the inputs combine their partial minima with
// an exact floating-point atomic min.
// --------------------------------------------------------------------------

// Packed pair of FP32 values and a packed subtraction rounded toward -inf
// (PTX sub.rm.f32x2, sm_100 and later).
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ unsigned long long pack2(double, double) { return 0ull; }
__device__ __forceinline__ void sub_rd_x2(unsigned long long a, unsigned long long b, float& lo,
                                          float& hi) {
    unsigned long long d;
    asm("sub.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(d));
}

template <typename T, int R, int TC, bool P2, bool PACKED>
__global__ void __launch_bounds__(256)
ctransform_kernel(const PairDev* __restrict__ pairs, const CtItem* __restrict__ items,
                  int n_items, int phase) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* hs = reinterpret_cast<T*>(smem_raw);
    constexpr int NQ = R + TC - 1;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const CtItem I = items[it];
        const PairDev& P = pairs[I.pair];
        const int N = P.N, m = P.m;
        const bool d3 = P.d == 3;
        const T* h = reinterpret_cast<const T*>(phase == 0 ? P.fhat : P.g);
        T* out = reinterpret_cast<T*>(phase == 0 ? P.g : P.f);
        const int nin = I.in_rows * N;
        const T* hsrc = h + (size_t)I.in_row0 * N;
        for (int k = threadIdx.x; k < nin; k += blockDim.x) hs[k] = hsrc[k];
        __syncthreads();
        const int o_end = min(I.out0 + CT_TILE, m);
        for (int o = I.out0 + threadIdx.x * R; o < o_end; o += blockDim.x * R) {
            T mins[R];
#pragma unroll
            for (int r = 0; r < R; ++r) mins[r] = pos_inf<T>();
            // a line of N points: every coordinate but the last is fixed
            // (2-D: the row j1; 3-D: (ja, jb)), j2 is the last coordinate
            const int j1 = o / N, j2 = o % N;
            const int ja = d3 ? j1 / N : j1, jb = d3 ? j1 % N : 0;
            const T* tab = reinterpret_cast<const T*>(P.ctab_lo);
            for (int c0 = 0; c0 < N; c0 += TC) {
                T colq[NQ];
                if constexpr (P2) {
#pragma unroll
                    for (int e = 0; e < NQ; ++e) {
                        const T d = (T)(c0 - j2 + e - (R - 1));
                        colq[e] = d * d;
                    }
                }
                for (int r1 = 0; r1 < I.in_rows; ++r1) {
                    const int i1 = I.in_row0 + r1;
                    const int ia = d3 ? i1 / N : i1, ib = d3 ? i1 % N : 0;
                    T q[NQ];
                    if constexpr (P2) {
                        const T A = (T)((ia - ja) * (ia - ja) + (ib - jb) * (ib - jb));
#pragma unroll
                        for (int e = 0; e < NQ; ++e) q[e] = A + colq[e];      // exact integers
                    } else {
                        const T* trow = tab + ((size_t)abs(ia - ja) * (d3 ? N : 1) + abs(ib - jb)) * N;
#pragma unroll
                        for (int e = 0; e < NQ; ++e) q[e] = trow[abs(c0 - j2 + e - (R - 1))];
                    }
                    T fv[TC];
                    const T* hrow = hs + r1 * N + c0;
#pragma unroll
                    for (int s = 0; s < TC; ++s) fv[s] = hrow[s];
                    if constexpr (PACKED && TC % 2 == 0 && sizeof(T) == 4) {
                        // two candidates per packed subtraction: (q_e, q_e+1) - (f_s, f_s+1)
                        // rounded toward -inf, then one 3-input min
                        unsigned long long qa[(NQ + 1) / 2], qb[NQ / 2], fp[TC / 2];
#pragma unroll
                        for (int j = 0; j < (NQ + 1) / 2; ++j)
                            qa[j] = pack2(q[2 * j], 2 * j + 1 < NQ ? q[2 * j + 1] : T(0));
#pragma unroll
                        for (int j = 0; j < NQ / 2; ++j)
                            qb[j] = pack2(q[2 * j + 1], 2 * j + 2 < NQ ? q[2 * j + 2] : T(0));
#pragma unroll
                        for (int j = 0; j < TC / 2; ++j) fp[j] = pack2(fv[2 * j], fv[2 * j + 1]);
#pragma unroll
                        for (int s = 0; s < TC; s += 2)
#pragma unroll
                            for (int r = 0; r < R; ++r) {
                                const int e = s - r + R - 1;
                                const unsigned long long qq = (e % 2 == 0) ? qa[e / 2] : qb[e / 2];
                                float t0, t1;
                                sub_rd_x2(qq, fp[s / 2], t0, t1);
                                mins[r] = min3(mins[r], t0, t1);
                            }
                    } else if constexpr (TC % 2 == 0) {
#pragma unroll
                        for (int s = 0; s < TC; s += 2)
#pragma unroll
                            for (int r = 0; r < R; ++r)
                                mins[r] = min3(mins[r], sub_rd(q[s - r + R - 1], fv[s]),
                                               sub_rd(q[s + 1 - r + R - 1], fv[s + 1]));
                    } else {
#pragma unroll
                        for (int s = 0; s < TC; ++s)
#pragma unroll
                            for (int r = 0; r < R; ++r)
                                mins[r] = fmin(mins[r], sub_rd(q[s - r + R - 1], fv[s]));
                    }
                }
            }
            if (I.in_rows < P.rows) {      // partial minimum: combine across items
#pragma unroll
                for (int r = 0; r < R; ++r) atomic_min_fp(&out[o + r], mins[r]);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) out[o + r] = mins[r];
            }
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------------------
// Line-paired variant (FP32): the same candidates, packed two input lines at
// a time.  For input lines i1, i1' and output j, the candidates
// c(i1, s; j) - h(i1, s) and c(i1', s; j) - h(i1', s) share the column offset
// s - j2, so one packed subtraction rounded toward -inf (sub.rm.f32x2) forms
// both and one 3-input min folds both into out_j.  The staged inputs are
// interleaved by line pairs, (h(i1, c), h(i1', c)), so one 16-byte shared
// load brings two packed operands.  The packed costs (A + D_e, A' + D_e) are
// one packed addition of the line parts (A, A') and the duplicated column
// part (D_e, D_e) (exact integers for p = 2), computed when first needed: for
// the column s the R outputs use the costs e = s .. s + R - 1, a window that
// slides by one per column.  Per two candidates this issues one packed
// subtraction and one 3-input min.  An odd last line is paired with
// h = -inf, whose candidates are +inf.
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long add_rn_x2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// m' = min(m, fl_down(w.lo - h.lo), fl_down(w.hi - h.hi)) in one assembly block
__device__ __forceinline__ float sub2_min3(unsigned long long w, unsigned long long h, float m) {
    float d;
    asm("{\n .reg .b64 t;\n .reg .f32 lo, hi;\n sub.rm.f32x2 t, %1, %2;\n mov.b64 {lo, hi}, t;\n"
        " min.f32 %0, %3, lo, hi;\n}"
        : "=f"(d) : "l"(w), "l"(h), "f"(m));
    return d;
}
__device__ __forceinline__ unsigned long long fma_rn_x2(unsigned long long a, unsigned long long b,
                                                        unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// MINB: resident CTAs per SM the register budget is cut for (1: no cut).
// DDFLY (p = 2): form each new window cost from a packed (d, d) pair as
// fma(d, d, A), d advancing by one per column, instead of keeping the NQ
// squared column offsets of a chunk in registers (fewer registers, one more
// FMA-pipe instruction per new cost).
// FUSE: the staged h pairs are read as two 64-bit operands per 16-byte load,
// and each candidate pair's packed subtraction and 3-input min are one inline
// assembly block, so no value crosses between the packed and the scalar views
// outside it.
template <int R, int TC, bool P2, bool D3, int MINB = 1, bool DDFLY = false, bool FUSE = false>
__global__ void __launch_bounds__(256, MINB)
ctransform_rp_kernel(const PairDev* __restrict__ pairs, const CtItem* __restrict__ items,
                     int n_items, int phase) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* hs2 = reinterpret_cast<float2*>(smem_raw);      // [line pair][column]
    constexpr int NQ = R + TC - 1;
    static_assert(TC % 2 == 0, "two columns per 16-byte shared load");
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const CtItem I = items[it];
        const PairDev& P = pairs[I.pair];
        const int N = P.N, m = P.m;
        const float* h = reinterpret_cast<const float*>(phase == 0 ? P.fhat : P.g);
        float* out = reinterpret_cast<float*>(phase == 0 ? P.g : P.f);
        const int npairs = (I.in_rows + 1) >> 1;
        const float* hsrc = h + (size_t)I.in_row0 * N;
        for (int k = threadIdx.x; k < npairs * N; k += blockDim.x) {
            const int lp = k / N, c = k - lp * N;
            const float lo = hsrc[(size_t)(2 * lp) * N + c];
            const float hi = 2 * lp + 1 < I.in_rows ? hsrc[(size_t)(2 * lp + 1) * N + c]
                                                    : __int_as_float(0xff800000);   // -inf
            hs2[k] = make_float2(lo, hi);
        }
        __syncthreads();
        const float* refl = reinterpret_cast<const float*>(P.ctab_lo_refl);
        const int o_end = min(I.out0 + CT_TILE, m);
        const int last = I.in_row0 + I.in_rows - 1;
        for (int o = I.out0 + threadIdx.x * R; o < o_end; o += blockDim.x * R) {
            float mins[R];
#pragma unroll
            for (int r = 0; r < R; ++r) mins[r] = pos_inf<float>();
            const int j1 = o / N, j2 = o % N;
            const int ja = D3 ? j1 / N : j1, jb = D3 ? j1 % N : 0;
            for (int c0 = 0; c0 < N; c0 += TC) {
                unsigned long long DD[(P2 && !DDFLY) ? NQ : 1];   // (D_e, D_e), p = 2
                if constexpr (P2 && !DDFLY) {
#pragma unroll
                    for (int e = 0; e < NQ; ++e) {
                        const float d = (float)(c0 - j2 + e - (R - 1));
                        DD[e] = pack2(d * d, d * d);
                    }
                }
                // DDFLY: (d, d) of cost e = 0; each new cost advances it by one
                const unsigned long long dd0 = pack2((float)(c0 - j2 - (R - 1)), (float)(c0 - j2 - (R - 1)));
                const float4* hrow = reinterpret_cast<const float4*>(hs2 + c0);
                int i1 = I.in_row0;
                for (int lp = 0; lp < npairs; ++lp, hrow += N / 2, i1 += 2) {
                    const int i1b = min(i1 + 1, last);          // odd tail: h = -inf there
                    unsigned long long AA = 0ull;
                    const float* t0 = nullptr;
                    const float* t1 = nullptr;
                    float tq0[P2 ? 1 : ((NQ + 3) / 4) * 4], tq1[P2 ? 1 : ((NQ + 3) / 4) * 4];
                    if constexpr (P2) {
                        float A1, A2;
                        if constexpr (D3) {
                            const int ia = i1 / N, ib = i1 - (i1 / N) * N;
                            const int ia2 = i1b / N, ib2 = i1b - (i1b / N) * N;
                            A1 = (float)((ia - ja) * (ia - ja) + (ib - jb) * (ib - jb));
                            A2 = (float)((ia2 - ja) * (ia2 - ja) + (ib2 - jb) * (ib2 - jb));
                        } else {
                            A1 = (float)((i1 - ja) * (i1 - ja));
                            A2 = (float)((i1b - ja) * (i1b - ja));
                        }
                        AA = pack2(A1, A2);
                    } else {
                        // reflected table rows: row[c + N - 1] = table[|c|]; the
                        // chunk's costs are NQ consecutive entries from an
                        // offset that is a multiple of 8 floats
                        size_t r0, r1;
                        if constexpr (D3) {
                            const int ia = i1 / N, ib = i1 - (i1 / N) * N;
                            const int ia2 = i1b / N, ib2 = i1b - (i1b / N) * N;
                            r0 = (size_t)abs(ia - ja) * N + abs(ib - jb);
                            r1 = (size_t)abs(ia2 - ja) * N + abs(ib2 - jb);
                        } else {
                            r0 = (size_t)abs(i1 - ja);
                            r1 = (size_t)abs(i1b - ja);
                        }
                        const int off = c0 - j2 - (R - 1) + N - 1;
                        t0 = refl + r0 * (2 * N) + off;
                        t1 = refl + r1 * (2 * N) + off;
#pragma unroll
                        for (int q = 0; q < (NQ + 3) / 4; ++q) {
                            const float4 u = reinterpret_cast<const float4*>(t0)[q];
                            const float4 w = reinterpret_cast<const float4*>(t1)[q];
                            tq0[4 * q] = u.x; tq0[4 * q + 1] = u.y; tq0[4 * q + 2] = u.z; tq0[4 * q + 3] = u.w;
                            tq1[4 * q] = w.x; tq1[4 * q + 1] = w.y; tq1[4 * q + 2] = w.z; tq1[4 * q + 3] = w.w;
                        }
                    }
                    unsigned long long dd = dd0;                // DDFLY: (d_e, d_e) of the next cost
                    // costs are requested in increasing e (0, 1, ..., NQ - 1)
                    auto cost = [&](int e) -> unsigned long long {
                        if constexpr (P2 && DDFLY) {
                            const unsigned long long c = fma_rn_x2(dd, dd, AA);   // d^2 + A, exact integers
                            dd = add_rn_x2(dd, 0x3f8000003f800000ull);           // d + 1 (both halves)
                            return c;
                        } else if constexpr (P2) {
                            return add_rn_x2(AA, DD[e]);            // exact integers
                        } else {
                            return pack2(tq0[e], tq1[e]);
                        }
                    };
                    // window of costs for column s: e = s - r + R - 1, r = R-1 .. 0
                    // before column 0 the window is that of column -1: win[r] = cost(R - 2 - r)
                    unsigned long long win[R];
#pragma unroll
                    for (int r = R - 2; r >= 0; --r) win[r] = cost(R - 2 - r);
#pragma unroll
                    for (int s = 0; s < TC; s += 2) {
                        unsigned long long hp0, hp1;
                        if constexpr (FUSE) {
                            const ulonglong2 v = reinterpret_cast<const ulonglong2*>(hrow)[s / 2];
                            hp0 = v.x; hp1 = v.y;
                        } else {
                            const float4 v = hrow[s / 2];
                            hp0 = pack2(v.x, v.y); hp1 = pack2(v.z, v.w);
                        }
#pragma unroll
                        for (int ss = 0; ss < 2; ++ss) {
                            const int sc = s + ss;
                            // slide: win[r] holds cost e = sc - r + R - 1
#pragma unroll
                            for (int r = R - 1; r > 0; --r) win[r] = win[r - 1];
                            win[0] = cost(sc + R - 1);
                            const unsigned long long hp = ss ? hp1 : hp0;
#pragma unroll
                            for (int r = 0; r < R; ++r) {
                                if constexpr (FUSE) {
                                    mins[r] = sub2_min3(win[r], hp, mins[r]);
                                } else {
                                    float a, b;
                                    sub_rd_x2(win[r], hp, a, b);
                                    mins[r] = min3(mins[r], a, b);
                                }
                            }
                        }
                    }
                }
            }
            if (I.in_rows < P.rows) {
#pragma unroll
                for (int r = 0; r < R; ++r) atomic_min_fp(&out[o + r], mins[r]);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) out[o + r] = mins[r];
            }
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------------------
// Shifted line-paired variant (p = 2, FP32, 2-D).  With c_ij = A + D,
// A = (i1 - j1)^2 the line part and D = (i2 - j2)^2 the column part, the
// candidate is c_ij - h_i = D - (h_i - A).  Per input line pair the thread
// forms hA = h - A once per staged value, rounded up (so hA >= h - A), and
// every candidate of the pair is fl_down(D_e - hA) with the column parts D_e
// of the chunk's window, which do not depend on the line: one packed
// subtraction and one 3-input min per two candidates, no per-line window.
// Since D - hA <= c - h, every candidate is at most the exact c_ij - h_i and
// h_i + out_j <= c_ij holds exactly; against the transform rounded down once
// per candidate, a result can be lower by the rounding of hA (an ulp of
// |h - A|).  A odd last line is paired with h = -inf (candidates +inf).
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long sub_ru_x2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rp.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long mul_rn_x2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// PIN: the chunk's squared column offsets pass through a volatile move when
// they are formed, so that the compiler keeps them in registers across the
// line-pair loop instead of forming them again inside it.
__device__ __forceinline__ unsigned long long pin64(unsigned long long v) {
    unsigned long long r;
    asm volatile("mov.b64 %0, %1;" : "=l"(r) : "l"(v));
    return r;
}

template <int R, int TC, int MINB, bool PIN = false>
__global__ void __launch_bounds__(256, MINB)
ctransform_rpd_kernel(const PairDev* __restrict__ pairs, const CtItem* __restrict__ items,
                      int n_items, int phase) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* hs2 = reinterpret_cast<float2*>(smem_raw);      // [line pair][column]
    constexpr int NQ = R + TC - 1;
    static_assert(TC % 2 == 0, "two columns per 16-byte shared load");
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const CtItem I = items[it];
        const PairDev& P = pairs[I.pair];
        const int N = P.N, m = P.m;
        const float* h = reinterpret_cast<const float*>(phase == 0 ? P.fhat : P.g);
        float* out = reinterpret_cast<float*>(phase == 0 ? P.g : P.f);
        const int npairs = (I.in_rows + 1) >> 1;
        const float* hsrc = h + (size_t)I.in_row0 * N;
        for (int k = threadIdx.x; k < npairs * N; k += blockDim.x) {
            const int lp = k / N, c = k - lp * N;
            const float lo = hsrc[(size_t)(2 * lp) * N + c];
            const float hi = 2 * lp + 1 < I.in_rows ? hsrc[(size_t)(2 * lp + 1) * N + c]
                                                    : __int_as_float(0xff800000);   // -inf
            hs2[k] = make_float2(lo, hi);
        }
        __syncthreads();
        const int o_end = min(I.out0 + CT_TILE, m);
        for (int o = I.out0 + threadIdx.x * R; o < o_end; o += blockDim.x * R) {
            float mins[R];
#pragma unroll
            for (int r = 0; r < R; ++r) mins[r] = pos_inf<float>();
            const int j1 = o / N, j2 = o % N;
            const float a0 = (float)(I.in_row0 - j1);                 // i1 - j1 of the first line
            for (int c0 = 0; c0 < N; c0 += TC) {
                unsigned long long DD[NQ];                            // (D_e, D_e), exact integers
#pragma unroll
                for (int e = 0; e < NQ; ++e) {
                    const float d = (float)(c0 - j2 + e - (R - 1));
                    DD[e] = PIN ? pin64(pack2(d * d, d * d)) : pack2(d * d, d * d);
                }
                const ulonglong2* hrow = reinterpret_cast<const ulonglong2*>(hs2 + c0);
                unsigned long long tt = pack2(a0, a0 + 1.0f);         // (i1 - j1, i1 + 1 - j1)
                for (int lp = 0; lp < npairs; ++lp, hrow += N / 2) {
                    const unsigned long long AA = mul_rn_x2(tt, tt);  // line parts, exact
                    tt = add_rn_x2(tt, 0x4000000040000000ull);        // + (2, 2)
#pragma unroll
                    for (int s = 0; s < TC; s += 2) {
                        const ulonglong2 v = hrow[s / 2];
                        const unsigned long long hA0 = sub_ru_x2(v.x, AA), hA1 = sub_ru_x2(v.y, AA);
#pragma unroll
                        for (int ss = 0; ss < 2; ++ss) {
                            const unsigned long long hA = ss ? hA1 : hA0;
#pragma unroll
                            for (int r = 0; r < R; ++r) mins[r] = sub2_min3(DD[s + ss - r + R - 1], hA, mins[r]);
                        }
                    }
                }
            }
            if (I.in_rows < P.rows) {
#pragma unroll
                for (int r = 0; r < R; ++r) atomic_min_fp(&out[o + r], mins[r]);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) out[o + r] = mins[r];
            }
        }
        __syncthreads();
    }
}

template <int R, int TC, int MINB, bool PIN = false>
static int ct_launch_rpd(const PairDev* pairs_d, const CtItem* items, int n_items, int phase,
                         int threads, int in_rows, int N_max, int grid_cap, cudaStream_t stream) {
    auto kern = ctransform_rpd_kernel<R, TC, MINB, PIN>;
    threads = std::min(threads, CT_TILE / R);
    const size_t smem = sizeof(float2) * (size_t)((in_rows + 1) / 2) * N_max;
    if (smem > 227 * 1024) return QWB_ERR_UNSUPPORTED;
    QWB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int grid = n_items;
    if (grid_cap > 0) {
        int occ = 1;
        QWB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem));
        grid = std::min(n_items, grid_cap * std::max(1, occ));
    }
    kern<<<grid, threads, smem, stream>>>(pairs_d, items, n_items, phase);
    QWB_LAUNCHED();
    return QWB_OK;
}

int ct_pick_r(int N, int want) {
    for (int r = want; r > 1; r >>= 1)
        if (N % r == 0) return r;
    return 1;
}

template <typename T, int R, int TC, bool P2, bool PK>
static int ct_launch_rt(const PairDev* pairs_d, const CtItem* items, int n_items, int phase,
                        int threads, int in_rows, int N_max, int grid_cap, cudaStream_t stream) {
    auto kern = ctransform_kernel<T, R, TC, P2, PK>;
    const size_t smem = sizeof(T) * (size_t)in_rows * N_max;
    if (smem > 227 * 1024) return QWB_ERR_UNSUPPORTED;
    QWB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // persistent form: grid_cap = SM count; as many CTAs as fit at once
    int grid = n_items;
    if (grid_cap > 0) {
        int occ = 1;
        QWB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem));
        grid = std::min(n_items, grid_cap * std::max(1, occ));
    }
    kern<<<grid, threads, smem, stream>>>(pairs_d, items, n_items, phase);
    QWB_LAUNCHED();
    return QWB_OK;
}

template <int R, int TC, bool P2>
static int ct_launch_rp(const PairDev* pairs_d, const CtItem* items, int n_items, int phase,
                        int threads, int in_rows, int N_max, int grid_cap, bool d3,
                        cudaStream_t stream) {
    auto kern = d3 ? ctransform_rp_kernel<R, TC, P2, true> : ctransform_rp_kernel<R, TC, P2, false>;
    threads = std::min(threads, CT_TILE / R);     // every thread owns R outputs of the tile
    const size_t smem = sizeof(float2) * (size_t)((in_rows + 1) / 2) * N_max;
    if (smem > 227 * 1024) return QWB_ERR_UNSUPPORTED;
    QWB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int grid = n_items;
    if (grid_cap > 0) {
        int occ = 1;
        QWB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem));
        grid = std::min(n_items, grid_cap * std::max(1, occ));
    }
    kern<<<grid, threads, smem, stream>>>(pairs_d, items, n_items, phase);
    QWB_LAUNCHED();
    return QWB_OK;
}

template <int R, int TC, bool P2, int MINB, bool DDFLY, bool FUSE = false>
static int ct_launch_rp2d(const PairDev* pairs_d, const CtItem* items, int n_items, int phase,
                          int threads, int in_rows, int N_max, int grid_cap, cudaStream_t stream) {
    auto kern = ctransform_rp_kernel<R, TC, P2, false, MINB, DDFLY, FUSE>;
    threads = std::min(threads, CT_TILE / R);
    const size_t smem = sizeof(float2) * (size_t)((in_rows + 1) / 2) * N_max;
    if (smem > 227 * 1024) return QWB_ERR_UNSUPPORTED;
    QWB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int grid = n_items;
    if (grid_cap > 0) {
        int occ = 1;
        QWB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem));
        grid = std::min(n_items, grid_cap * std::max(1, occ));
    }
    kern<<<grid, threads, smem, stream>>>(pairs_d, items, n_items, phase);
    QWB_LAUNCHED();
    return QWB_OK;
}

template <typename T, bool P2>
static int ct_launch_t(const PairDev* pairs_d, const CtItem* items, int n_items, int phase,
                       const CtConfig& c, int N_max, int grid_cap, cudaStream_t stream) {
#define QWB_CT(RR, TT, PK)                                                                 \
    if (c.R == RR && c.TC == TT && c.packed == PK)                                         \
        return ct_launch_rt<T, RR, TT, P2, (PK != 0)>(pairs_d, items, n_items, phase, c.threads,  \
                                               c.in_rows, N_max, grid_cap, stream);
    QWB_CT(1, 1, 0) QWB_CT(2, 2, 0) QWB_CT(4, 4, 0) QWB_CT(8, 8, 0)
    QWB_CT(16, 8, 0) QWB_CT(16, 16, 0) QWB_CT(8, 16, 0)
    QWB_CT(8, 8, 1) QWB_CT(16, 8, 1) QWB_CT(16, 16, 1)
#undef QWB_CT
    if constexpr (sizeof(T) == 4) {
#define QWB_CTRP(RR, TT)                                                                   \
        if (c.R == RR && c.TC == TT && c.packed == 2)                                      \
            return ct_launch_rp<RR, TT, P2>(pairs_d, items, n_items, phase, c.threads,     \
                                            c.in_rows, N_max, grid_cap, c.has_3d, stream);
        QWB_CTRP(8, 8) QWB_CTRP(16, 8) QWB_CTRP(8, 16) QWB_CTRP(16, 16)
#undef QWB_CTRP
        // packings 3-6 (2-D only): line pairs with the register budget cut for
        // MINB resident CTAs per SM; DDFLY: p = 2 window costs formed on the fly
        if (c.packed >= 3 && c.packed <= 6 && c.has_3d) return QWB_ERR_UNSUPPORTED;
#define QWB_CTRPV(PK, MB, FLY, RR, TT)                                                     \
        if (c.R == RR && c.TC == TT && c.packed == PK)                                     \
            return ct_launch_rp2d<RR, TT, P2, MB, (P2 && FLY)>(pairs_d, items, n_items, phase, \
                                                            c.threads, c.in_rows, N_max, grid_cap, stream);
        QWB_CTRPV(3, 3, true, 8, 8)
        QWB_CTRPV(4, 3, false, 8, 8) QWB_CTRPV(4, 3, false, 8, 16)
        QWB_CTRPV(5, 2, false, 8, 16) QWB_CTRPV(5, 2, false, 16, 8) QWB_CTRPV(5, 2, false, 16, 16)
        QWB_CTRPV(6, 2, true, 8, 16)
#undef QWB_CTRPV
        // packings 7, 8 (2-D only): packings 5 and 2 with the fused
        // subtraction-and-min blocks
        if ((c.packed == 7 || c.packed == 8) && c.has_3d) return QWB_ERR_UNSUPPORTED;
#define QWB_CTRPF(PK, MB, RR, TT)                                                          \
        if (c.R == RR && c.TC == TT && c.packed == PK)                                     \
            return ct_launch_rp2d<RR, TT, P2, MB, false, true>(pairs_d, items, n_items, phase, \
                                                            c.threads, c.in_rows, N_max, grid_cap, stream);
        QWB_CTRPF(7, 2, 16, 16) QWB_CTRPF(7, 2, 16, 8) QWB_CTRPF(7, 2, 8, 16)
        QWB_CTRPF(8, 1, 16, 16)
#undef QWB_CTRPF
        // packings 9, 10 (p = 2, 2-D only): the shifted line-paired kernel with
        // the register budget of 2 (9) or 1 (10) resident CTAs per SM
        // packings 11, 12 (p = 2, 2-D only): 9 and 10 with the squared column
        // offsets pinned in registers
        if (c.packed >= 9 && c.packed <= 12 && (c.has_3d || !P2)) return QWB_ERR_UNSUPPORTED;
        if constexpr (P2) {
#define QWB_CTRPD(PK, MB, PIN, RR, TT)                                                     \
            if (c.R == RR && c.TC == TT && c.packed == PK)                                 \
                return ct_launch_rpd<RR, TT, MB, PIN>(pairs_d, items, n_items, phase, c.threads, c.in_rows, \
                                                      N_max, grid_cap, stream);
            QWB_CTRPD(9, 2, false, 16, 16) QWB_CTRPD(9, 2, false, 16, 8) QWB_CTRPD(9, 2, false, 8, 16)
            QWB_CTRPD(10, 1, false, 16, 16) QWB_CTRPD(10, 1, false, 32, 16) QWB_CTRPD(10, 1, false, 32, 8)
            QWB_CTRPD(11, 2, true, 16, 16) QWB_CTRPD(11, 2, true, 16, 8) QWB_CTRPD(11, 2, true, 8, 16)
            QWB_CTRPD(12, 1, true, 16, 16) QWB_CTRPD(12, 1, true, 32, 8)
#undef QWB_CTRPD
        }
    }
    return QWB_ERR_UNSUPPORTED;
}

int launch_ctransform(const PairDev* pairs_d, const CtItem* items, int n_items, int phase,
                      const CtConfig& cfg, int N_max, bool f64, int grid_cap, cudaStream_t stream) {
    if (n_items <= 0) return QWB_OK;
    // the p = 2 specialisation needs every pair of the launch at p = 2
    const bool p2 = cfg.p2;
    const CtConfig& c = cfg;
    if (f64) return p2 ? ct_launch_t<double, true>(pairs_d, items, n_items, phase, c, N_max, grid_cap, stream)
                       : ct_launch_t<double, false>(pairs_d, items, n_items, phase, c, N_max, grid_cap, stream);
    return p2 ? ct_launch_t<float, true>(pairs_d, items, n_items, phase, c, N_max, grid_cap, stream)
              : ct_launch_t<float, false>(pairs_d, items, n_items, phase, c, N_max, grid_cap, stream);
}


}  // namespace qwb
