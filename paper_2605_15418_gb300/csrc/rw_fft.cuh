// Shared-memory 2D FFT of one D x D complex patch, FP32, whole CTA.
//
// Mixed-radix Stockham autosort (radix 2, 3, 4, 8): stage with radix R after
// sub-transforms of length P reads x[i + q N/R], multiplies by
// exp(-+2 pi i q (i mod P) / (P R)), does a length-R DFT and writes
// y[(i / P) P R + (i mod P) + q P]; the output comes out in natural order.
// Each stage is done in place: all butterflies of the CTA are loaded into
// registers, the CTA synchronises, then they are stored.
//
// Layout: an N x N patch buffer keeps row b at X + b (N + 1).  With the odd
// row stride, and consecutive threads on consecutive rows (row pass) or
// columns (column pass), every load and store of a stage touches 16
// different bank pairs per half-warp: no shared-memory bank conflicts.
#pragma once
#include "rw_device.cuh"

template <int N>
struct Patch {
    static constexpr int S = N + 1;          // row stride (complex elements)
    // buffer size: also holds N rows of N + 2 samples staged by bulk copies
    static constexpr int ELEMS = N * (N + 2);
};

template <int R, bool INV>
__device__ __forceinline__ void dft_small(float2* u);

// 8-point DFT as two 4-point DFTs of the even and odd samples:
// y_k = E_k + W^k O_k, y_{k+4} = E_k - W^k O_k, W = exp(-+2 pi i / 8).
template <bool INV>
__device__ __forceinline__ void dft8(float2* u) {
    float2 e[4] = {u[0], u[2], u[4], u[6]};
    float2 o[4] = {u[1], u[3], u[5], u[7]};
    dft_small<4, INV>(e);
    dft_small<4, INV>(o);
    const float h = 0.70710678118654752440f;
    // W^1 o1, W^2 o2, W^3 o3 (forward W = (1 - i)/sqrt2; inverse conjugate)
    const float sg = INV ? 1.f : -1.f;
    const float2 w1 = make_float2(h * (o[1].x - sg * o[1].y), h * (o[1].y + sg * o[1].x));
    const float2 w2 = make_float2(-sg * o[2].y, sg * o[2].x);
    const float2 w3 = make_float2(h * (-o[3].x - sg * o[3].y), h * (-o[3].y + sg * o[3].x));
    u[0] = cadd(e[0], o[0]); u[4] = csub(e[0], o[0]);
    u[1] = cadd(e[1], w1);   u[5] = csub(e[1], w1);
    u[2] = cadd(e[2], w2);   u[6] = csub(e[2], w2);
    u[3] = cadd(e[3], w3);   u[7] = csub(e[3], w3);
}

template <int R, bool INV>
__device__ __forceinline__ void dft_small(float2* u) {
    if constexpr (R == 8) {
        dft8<INV>(u);
    } else if constexpr (R == 2) {
        float2 a = u[0], b = u[1];
        u[0] = cadd(a, b);
        u[1] = csub(a, b);
    } else if constexpr (R == 4) {
        float2 a = u[0], b = u[1], c = u[2], d = u[3];
        float2 s0 = cadd(a, c), s1 = csub(a, c), s2 = cadd(b, d), s3 = csub(b, d);
        // forward: y1 = s1 - i s3, y3 = s1 + i s3 ; inverse swaps
        float2 is3 = INV ? make_float2(-s3.y, s3.x) : make_float2(s3.y, -s3.x);  // -+ i s3
        u[0] = cadd(s0, s2);
        u[2] = csub(s0, s2);
        u[1] = cadd(s1, is3);
        u[3] = csub(s1, is3);
    } else if constexpr (R == 3) {
        const float c1 = -0.5f;
        const float s1 = INV ? 0.86602540378443864676f : -0.86602540378443864676f;
        float2 a = u[0], b = u[1], c = u[2];
        float2 t = cadd(b, c), d = csub(b, c);
        u[0] = cadd(a, t);
        float2 m = make_float2(a.x + c1 * t.x, a.y + c1 * t.y);
        // +- i s1 (b - c)
        float2 id = make_float2(-s1 * d.y, s1 * d.x);
        u[1] = cadd(m, id);
        u[2] = csub(m, id);
    }
}

// Line b and butterfly i of the k-th butterfly a thread owns in a stage.
// Row passes that divide evenly keep one butterfly index i per thread (its
// twiddles are loaded once) over PER rows BL apart, BL >= 16 consecutive
// threads on consecutive rows; otherwise (and in column passes, where this
// costs fewer registers overall) thread f works on line f % N, butterfly f / N.
template <int N, int NB, int PER, bool COLS>
struct StageMap {
    static constexpr int TOT = N * NB;
    static constexpr int BL = N / PER;
    static constexpr bool BLOCKED = (TOT % RW_THREADS == 0) && (N % PER == 0) &&
                                    (BL * NB == RW_THREADS) && (BL >= 16) && !COLS;
    __device__ static __forceinline__ void at(int k, int& b, int& i) {
        if constexpr (BLOCKED) {
            b = (int)threadIdx.x % BL + k * BL;
            i = (int)threadIdx.x / BL;
        } else {
            const int f = (int)threadIdx.x + k * RW_THREADS;
            b = f % N;
            i = f / N;
        }
    }
};

// One Stockham stage over all N rows (COLS = false) or all N columns.
template <int N, int R, int P, bool INV, bool COLS>
__device__ __forceinline__ void fft_stage(float2* buf, const float2* tw) {
    constexpr int S = Patch<N>::S;
    constexpr int NB = N / R;
    constexpr int TOT = N * NB;
    constexpr int PER = (TOT + RW_THREADS - 1) / RW_THREADS;
    using Map = StageMap<N, NB, PER, COLS>;
    float2 v[PER][R];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int f = threadIdx.x + k * RW_THREADS;
        if ((TOT % RW_THREADS == 0) || f < TOT) {
            int b, i;
            Map::at(k, b, i);
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int e = i + q * NB;
                v[k][q] = COLS ? buf[e * S + b] : buf[b * S + e];
            }
            if constexpr (P > 1) {
                const int kk = i % P;
#pragma unroll
                for (int q = 1; q < R; ++q) {
                    float2 w = tw[q * kk * (N / (P * R))];
                    if (INV) w.y = -w.y;
                    v[k][q] = cmul(v[k][q], w);
                }
            }
            dft_small<R, INV>(v[k]);
        }
    }
    main_sync();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int f = threadIdx.x + k * RW_THREADS;
        if ((TOT % RW_THREADS == 0) || f < TOT) {
            int b, i;
            Map::at(k, b, i);
            const int kk = i % P;
            const int j = (i / P) * P * R + kk;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const int e = j + q * P;
                if (COLS) buf[e * S + b] = v[k][q]; else buf[b * S + e] = v[k][q];
            }
        }
    }
    main_sync();
}

template <int N, bool INV, bool COLS>
__device__ __forceinline__ void fft_pass(float2* buf, const float2* tw) {
    if constexpr (N == 16) {
        fft_stage<16, 4, 1, INV, COLS>(buf, tw);
        fft_stage<16, 4, 4, INV, COLS>(buf, tw);
    } else if constexpr (N == 32) {
        fft_stage<32, 4, 1, INV, COLS>(buf, tw);
        fft_stage<32, 8, 4, INV, COLS>(buf, tw);
    } else if constexpr (N == 64) {
        fft_stage<64, 8, 1, INV, COLS>(buf, tw);
        fft_stage<64, 8, 8, INV, COLS>(buf, tw);
    } else if constexpr (N == 96) {
        fft_stage<96, 8, 1, INV, COLS>(buf, tw);
        fft_stage<96, 4, 8, INV, COLS>(buf, tw);
        fft_stage<96, 3, 32, INV, COLS>(buf, tw);
    } else if constexpr (N == 128) {
        fft_stage<128, 8, 1, INV, COLS>(buf, tw);
        fft_stage<128, 4, 8, INV, COLS>(buf, tw);
        fft_stage<128, 4, 32, INV, COLS>(buf, tw);
    }
}

// First row stage (radix R, no twiddles) reading rows staged with stride
// N + 2 at column offset `off` and writing the usual stride N + 1 layout in
// place: every load of the stage happens before its barrier.
// Staged rows have the even stride N + 2 (16-byte aligned bulk copies), so
// the usual map (a warp on 32 consecutive rows, one butterfly) would put rows
// b and b + 8 of a half-warp on the same banks.  For N = 64, radix 8 a
// half-warp instead takes 8 consecutive rows x 2 adjacent butterflies:
// (4 b + 2 i) mod 32 then covers every bank once on the staged reads, and
// (2 b + 16 i) mod 32 on the stride N + 1 writes.
template <int N, int NB, int PER>
struct StagedMap {
    static constexpr bool SPLIT = (N == 64) && (NB == 8) && (N * NB == PER * RW_THREADS);
    __device__ static __forceinline__ void at(int k, int& b, int& i) {
        if constexpr (SPLIT) {
            const int f = ltid() + k * RW_THREADS;
            const int j = f & 15, hw = f >> 4;
            b = 8 * (hw & 7) + (j >> 1);
            i = 2 * (hw >> 3) + (j & 1);
        } else {
            StageMap<N, NB, PER, false>::at(k, b, i);
        }
    }
};

template <int N, int R, bool INV>
__device__ __forceinline__ void fft_stage_from_staged(float2* buf, int off) {
    constexpr int S = Patch<N>::S, SS = N + 2;
    constexpr int NB = N / R;
    constexpr int TOT = N * NB;
    constexpr int PER = (TOT + RW_THREADS - 1) / RW_THREADS;
    using Map = StagedMap<N, NB, PER>;
    float2 v[PER][R];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int f = threadIdx.x + k * RW_THREADS;
        if ((TOT % RW_THREADS == 0) || f < TOT) {
            int b, i;
            Map::at(k, b, i);
#pragma unroll
            for (int q = 0; q < R; ++q) v[k][q] = buf[b * SS + off + i + q * NB];
            dft_small<R, INV>(v[k]);
        }
    }
    main_sync();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int f = threadIdx.x + k * RW_THREADS;
        if ((TOT % RW_THREADS == 0) || f < TOT) {
            int b, i;
            Map::at(k, b, i);
#pragma unroll
            for (int q = 0; q < R; ++q) buf[b * S + i * R + q] = v[k][q];
        }
    }
    main_sync();
}

// 2D FFT of an N = 64 patch staged as rows of N + 2 samples (bulk copies),
// the patch starting at column `off` of each staged row.
template <int N, bool INV>
__device__ __forceinline__ void fft2d_staged(float2* buf, const float2* tw, int off) {
    static_assert(N == 64, "staged patches are 64 x 64");
    fft_stage_from_staged<64, 8, INV>(buf, off);
    fft_stage<64, 8, 8, INV, false>(buf, tw);
    fft_pass<64, INV, true>(buf, tw);
}

// X[b][a] -> sum_{a,b} X[b][a] exp(-+2 pi i (m_u a + m_v b) / N), natural
// order, X[b][a] at buf[b (N + 1) + a].
template <int N, bool INV>
__device__ __forceinline__ void fft2d(float2* buf, const float2* tw) {
    fft_pass<N, INV, false>(buf, tw);
    fft_pass<N, INV, true>(buf, tw);
}

// tw[t] = exp(-2 pi i t / N), t in [0, N).
template <int N>
__device__ __forceinline__ void fft_twiddles(float2* tw) {
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        float s, c;
        sincospif(-2.0f * (float)t / (float)N, &s, &c);
        tw[t] = make_float2(c, s);
    }
}
