// 3D Hessian action with thread-local quadrature columns (sm_103a).
//
// y = G^T B^T (H : B G v) (paper Sec. 3.4, eq. vm_pa_hess) for one element
// per MX x MX thread square.  A thread owning (q1, q2) keeps the nine
// reference-gradient components dA_{cb}(q1, q2, q3) of its q3 column in
// registers from the last forward contraction, through the pointwise product
// with the stored data, into the first transposed contraction, so no
// per-point array lives in shared memory: an element needs only the node
// block and the two intermediate tensors (384 values for p = 3), which keeps
// more elements resident per SM than the generic kernel.  Accumulations use
// the unnormalised acc_add (normalised once per stored value).
#pragma once

#include <type_traits>

#include "elem_kernels.cuh"

namespace tmop {

template <class C, class R>
struct Apply3Layout {
    static constexpr int TAB = 2 * C::NQ * C::NI;                       // B, G
    static constexpr int TAB_PAD = (TAB + 1) & ~1;
    static constexpr int SLOT = (C::SU + C::S1 + C::S2 + 1) & ~1;
    static constexpr size_t bytes = sizeof(R) * (size_t)(TAB_PAD + C::EPB * SLOT) +
                                    sizeof(int) * (size_t)(C::EPB * C::NP);
};

template <class C, class RV, class RC>
__device__ __forceinline__ void apply3_body(ElemParams P, const RV *__restrict__ v,
                                            const RC *__restrict__ H, RV *__restrict__ ev,
                                            const int *__restrict__ stop_iter, int k, BatchArgs BA)
{
    static_assert(C::D == 3, "3D kernel");
    constexpr int NI = C::NI, NQ = C::NQ, NP = C::NP, NQD = C::NQD, NS = C::NS;
    constexpr int O1 = NI * NI * NQ, O2 = NI * NQ * NQ;
    using L = Apply3Layout<C, RC>;
    const void *in = v, *aux = H;
    void *out = ev;
    const int *stop = stop_iter;
    const int64_t tile = resolve_tile(P, BA, in, aux, out, stop);
    v = static_cast<const RV *>(in);
    H = static_cast<const RC *>(aux);
    ev = static_cast<RV *>(out);
    if (stop && *stop < iter_of(stop, k)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    RC *base = reinterpret_cast<RC *>(smem);
    const RC *__restrict__ tab = table_of<RC>(P);
    for (int i = threadIdx.x; i < L::TAB; i += C::NT) base[i] = tab[i];
    const RC *B = base, *G = base + NQ * NI;
    const int slot = threadIdx.x / C::TPE;
    const bool act = slot < C::EPB;
    const int sl = act ? slot : 0;
    const int t = threadIdx.x - slot * C::TPE;
    const int tx = t % C::MX, ty = t / C::MX;
    RC *su = base + L::TAB_PAD + sl * L::SLOT;
    RC *s1 = su + C::SU;
    RC *s2 = s1 + C::S1;
    int *smap = reinterpret_cast<int *>(base + L::TAB_PAD + C::EPB * L::SLOT) + sl * NP;
    const int64_t e = tile * C::EPB + sl;
    const bool valid = act && e < P.E;
    if (valid)
        for (int i = t; i < NP; i += C::TPE) smap[i] = P.map[e * NP + i];
    __syncthreads();

    const bool qq = valid && tx < NQ && ty < NQ;     // owns a quadrature column
    RC col[9][NQ];                                   // dA_{cb} then Y_{cb} at (tx, ty, q3)

    // ---- forward: three contractions per component, the last into registers
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        if (valid)
            for (int i = t; i < NP; i += C::TPE) su[i] = RC(v[c * P.Nx + smap[i]]);
        __syncthreads();
        if (valid && tx < NQ && ty < NI) {
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                RC b = 0, g = 0;
#pragma unroll
                for (int i1 = 0; i1 < NI; ++i1) {
                    const RC u = su[(i3 * NI + ty) * NI + i1];
                    acc_add(b, B[tx * NI + i1] * u);
                    acc_add(g, G[tx * NI + i1] * u);
                }
                s1[(i3 * NI + ty) * NQ + tx] = norm(b);
                s1[O1 + (i3 * NI + ty) * NQ + tx] = norm(g);
            }
        }
        __syncthreads();
        if (qq) {
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                RC bb = 0, bg = 0, gb = 0;
#pragma unroll
                for (int i2 = 0; i2 < NI; ++i2) {
                    const RC sb = s1[(i3 * NI + i2) * NQ + tx];
                    const RC sg = s1[O1 + (i3 * NI + i2) * NQ + tx];
                    const RC Bq = B[ty * NI + i2], Gq = G[ty * NI + i2];
                    acc_add(bb, Bq * sb);
                    acc_add(bg, Gq * sb);
                    acc_add(gb, Bq * sg);
                }
                s2[(i3 * NQ + ty) * NQ + tx] = norm(gb);
                s2[O2 + (i3 * NQ + ty) * NQ + tx] = norm(bg);
                s2[2 * O2 + (i3 * NQ + ty) * NQ + tx] = norm(bb);
            }
        }
        __syncthreads();
        if (qq) {
            RC c0[NI], c1[NI], c2[NI];
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                c0[i3] = s2[(i3 * NQ + ty) * NQ + tx];
                c1[i3] = s2[O2 + (i3 * NQ + ty) * NQ + tx];
                c2[i3] = s2[2 * O2 + (i3 * NQ + ty) * NQ + tx];
            }
#pragma unroll
            for (int q3 = 0; q3 < NQ; ++q3) {
                RC r0 = 0, r1 = 0, r2 = 0;
#pragma unroll
                for (int i3 = 0; i3 < NI; ++i3) {
                    const RC Bq = B[q3 * NI + i3], Gq = G[q3 * NI + i3];
                    acc_add(r0, Bq * c0[i3]);
                    acc_add(r1, Bq * c1[i3]);
                    acc_add(r2, Gq * c2[i3]);
                }
                // component c is constant inside this unrolled body per c value
#pragma unroll
                for (int cc = 0; cc < 3; ++cc)
                    if (cc == c) {
                        col[cc * 3 + 0][q3] = norm(r0);
                        col[cc * 3 + 1][q3] = norm(r1);
                        col[cc * 3 + 2][q3] = norm(r2);
                    }
            }
        }
    }

    // ---- pointwise: Y = H : dA with the symmetric-packed stored data
    if (qq) {
        const RC *He = H + e * (int64_t)C::HST;
        const RC *Hc = He + (ty * NQ + tx);              // plain layout: the thread's column
#pragma unroll
        for (int q3 = 0; q3 < NQ; ++q3) {
            RC y[9];
#pragma unroll
            for (int r = 0; r < 9; ++r) y[r] = 0;
#pragma unroll
            for (int r = 0; r < 9; ++r)
#pragma unroll
                for (int s = r; s < 9; ++s) {
                    const RC h = C::PAIRS ? He[C::hoff(pidx<9>(r, s), q3 * NQ * NQ + ty * NQ + tx)]
                                          : Hc[pidx<9>(r, s) * NQD + q3 * NQ * NQ];
                    acc_add(y[r], h * col[s][q3]);
                    if (s != r) acc_add(y[s], h * col[r][q3]);
                }
#pragma unroll
            for (int r = 0; r < 9; ++r) col[r][q3] = norm(y[r]);
        }
    }

    // ---- transposed contractions per component, first one from registers
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        if (qq) {
            RC y0[NQ], y1[NQ], y2[NQ];
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
                if (cc == c) {
#pragma unroll
                    for (int q3 = 0; q3 < NQ; ++q3) {
                        y0[q3] = col[cc * 3 + 0][q3];
                        y1[q3] = col[cc * 3 + 1][q3];
                        y2[q3] = col[cc * 3 + 2][q3];
                    }
                }
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                RC z0 = 0, z1 = 0, z2 = 0;
#pragma unroll
                for (int q3 = 0; q3 < NQ; ++q3) {
                    const RC Bq = B[q3 * NI + i3], Gq = G[q3 * NI + i3];
                    acc_add(z0, Bq * y0[q3]);
                    acc_add(z1, Bq * y1[q3]);
                    acc_add(z2, Gq * y2[q3]);
                }
                s2[(i3 * NQ + ty) * NQ + tx] = norm(z0);
                s2[O2 + (i3 * NQ + ty) * NQ + tx] = norm(z1);
                s2[2 * O2 + (i3 * NQ + ty) * NQ + tx] = norm(z2);
            }
        }
        __syncthreads();
        if (valid && tx < NQ && ty < NI) {
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                RC a = 0, b = 0;
#pragma unroll
                for (int q2 = 0; q2 < NQ; ++q2) {
                    const RC Bq = B[q2 * NI + ty], Gq = G[q2 * NI + ty];
                    acc_add(a, Bq * s2[(i3 * NQ + q2) * NQ + tx]);
                    acc_add(b, Gq * s2[O2 + (i3 * NQ + q2) * NQ + tx]);
                    acc_add(b, Bq * s2[2 * O2 + (i3 * NQ + q2) * NQ + tx]);
                }
                s1[(i3 * NI + ty) * NQ + tx] = norm(a);
                s1[O1 + (i3 * NI + ty) * NQ + tx] = norm(b);
            }
        }
        __syncthreads();
        if (valid && tx < NI && ty < NI) {
            RV *out = ev + (int64_t)c * P.E * NP + e * NP;
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                RC o = 0;
#pragma unroll
                for (int q1 = 0; q1 < NQ; ++q1) {
                    acc_add(o, G[q1 * NI + tx] * s1[(i3 * NI + ty) * NQ + q1]);
                    acc_add(o, B[q1 * NI + tx] * s1[O1 + (i3 * NI + ty) * NQ + q1]);
                }
                ev_store(&out[(i3 * NI + ty) * NI + tx], norm(o));
            }
        }
    }
}

// The kernels.  FP32 data with n_q <= 4 runs 6 CTAs per SM (80 registers, no
// spills; the stored-data loads are latency-bound and more resident warps
// hide them: 48^3 Q3 0.428 -> 0.377 ms); every other configuration keeps the
// compiler's default register budget (an explicit minimum of one CTA per SM
// raised several configurations to ~255 registers and slowed them).  The
// double-float data at 4 CTAs per SM (128 registers, small spills) measured
// no faster (0.320 vs 0.33 of HBM).
template <class C, class RV, class RC>
__global__ void __launch_bounds__(C::NT)
k_apply3(ElemParams P, const RV *__restrict__ v, const RC *__restrict__ H, RV *__restrict__ ev,
         const int *__restrict__ stop_iter, int k, BatchArgs BA)
{
    apply3_body<C, RV, RC>(P, v, H, ev, stop_iter, k, BA);
}

template <class C, class RV, class RC>
__global__ void __launch_bounds__(C::NT, 6)
k_apply3_occ6(ElemParams P, const RV *__restrict__ v, const RC *__restrict__ H, RV *__restrict__ ev,
              const int *__restrict__ stop_iter, int k, BatchArgs BA)
{
    apply3_body<C, RV, RC>(P, v, H, ev, stop_iter, k, BA);
}

// ---------------------------------------------------------------------------
// The same action for many points per direction (the 9^3 rule): a q3 column
// of nine dA components no longer fits in registers, so the forward second
// stage of all three components stays in shared memory (9 NI NQ^2 values),
// each thread walks its q3 column point by point (dA from the shared stage
// values, Y = H : dA, and the first transposed contraction accumulated in
// registers), and the accumulators replace the stage values in place (a
// thread reads and writes only its own (q1, q2) entries, so no barrier is
// needed there).  About 34 KB of shared memory per element (p = 4, FP64
// class) against 89 KB for the generic kernel's per-point arrays.
template <class C, class R>
struct Apply3sLayout {
    static constexpr int O1 = C::NI * C::NI * C::NQ, O2 = C::NI * C::NQ * C::NQ;
    static constexpr int TAB = 2 * C::NQ * C::NI;
    static constexpr int TAB_PAD = (TAB + 1) & ~1;
    static constexpr int SLOT = (C::NP + 2 * O1 + 9 * O2 + 1) & ~1;
    static constexpr size_t bytes = sizeof(R) * (size_t)(TAB_PAD + C::EPB * SLOT) +
                                    sizeof(int) * (size_t)(C::EPB * C::NP);
};

template <class C, class RV, class RC>
__global__ void __launch_bounds__(C::NT, 4)
k_apply3s(ElemParams P, const RV *__restrict__ v, const RC *__restrict__ H, RV *__restrict__ ev,
          const int *__restrict__ stop_iter, int k, BatchArgs BA)
{
    static_assert(C::D == 3, "3D kernel");
    constexpr int NI = C::NI, NQ = C::NQ, NP = C::NP, NQD = C::NQD, NS = C::NS;
    using L = Apply3sLayout<C, RC>;
    constexpr int O1 = L::O1, O2 = L::O2;
    const void *in = v, *aux = H;
    void *out = ev;
    const int *stop = stop_iter;
    const int64_t tile = resolve_tile(P, BA, in, aux, out, stop);
    v = static_cast<const RV *>(in);
    H = static_cast<const RC *>(aux);
    ev = static_cast<RV *>(out);
    if (stop && *stop < iter_of(stop, k)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    RC *base = reinterpret_cast<RC *>(smem);
    const RC *__restrict__ tab = table_of<RC>(P);
    for (int i = threadIdx.x; i < L::TAB; i += C::NT) base[i] = tab[i];
    const RC *B = base, *G = base + NQ * NI;
    const int slot = threadIdx.x / C::TPE;
    const bool act = slot < C::EPB;
    const int sl = act ? slot : 0;
    const int t = threadIdx.x - slot * C::TPE;
    const int tx = t % C::MX, ty = t / C::MX;
    RC *su = base + L::TAB_PAD + sl * L::SLOT;
    RC *s1 = su + NP;
    RC *s2 = s1 + 2 * O1;          // [component c][stage output 0..2][O2]
    int *smap = reinterpret_cast<int *>(base + L::TAB_PAD + C::EPB * L::SLOT) + sl * NP;
    const int64_t e = tile * C::EPB + sl;
    const bool valid = act && e < P.E;
    if (valid)
        for (int i = t; i < NP; i += C::TPE) smap[i] = P.map[e * NP + i];
    __syncthreads();
    const bool qq = valid && tx < NQ && ty < NQ;
    const int col = ty * NQ + tx;

    // ---- forward: stages 1 and 2 of each component into s2[c]
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        if (valid)
            for (int i = t; i < NP; i += C::TPE) su[i] = RC(v[c * P.Nx + smap[i]]);
        __syncthreads();
        if (valid && tx < NQ && ty < NI) {
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                RC b = 0, g = 0;
#pragma unroll
                for (int i1 = 0; i1 < NI; ++i1) {
                    const RC u = su[(i3 * NI + ty) * NI + i1];
                    acc_add(b, B[tx * NI + i1] * u);
                    acc_add(g, G[tx * NI + i1] * u);
                }
                s1[(i3 * NI + ty) * NQ + tx] = norm(b);
                s1[O1 + (i3 * NI + ty) * NQ + tx] = norm(g);
            }
        }
        __syncthreads();
        if (qq) {
            RC *s2c = s2 + c * 3 * O2;
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                RC bb = 0, bg = 0, gb = 0;
#pragma unroll
                for (int i2 = 0; i2 < NI; ++i2) {
                    const RC sb = s1[(i3 * NI + i2) * NQ + tx];
                    const RC sg = s1[O1 + (i3 * NI + i2) * NQ + tx];
                    const RC Bq = B[ty * NI + i2], Gq = G[ty * NI + i2];
                    acc_add(bb, Bq * sb);
                    acc_add(bg, Gq * sb);
                    acc_add(gb, Bq * sg);
                }
                s2c[i3 * NQ * NQ + col] = norm(gb);
                s2c[O2 + i3 * NQ * NQ + col] = norm(bg);
                s2c[2 * O2 + i3 * NQ * NQ + col] = norm(bb);
            }
        }
        __syncthreads();      // su and s1 are reused by the next component
    }

    // ---- the thread's q3 column: dA, Y = H : dA, first transposed stage
    if (qq) {
        RC z[9][NI];
#pragma unroll
        for (int r = 0; r < 9; ++r)
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) z[r][i3] = 0;
        const RC *He = H + e * (int64_t)C::HST;
        const RC *Hc = He + col;                         // plain layout: the thread's column
        // FP32 data at p = 4: three points per iteration let the stored-data loads
        // of the next points overlap (no spills; 24^3 Kershaw p = 4 0.578 -> 0.537 ms
        // per action, no gain at p <= 3); double-float would spill
        constexpr int UQ = (std::is_same<RC, float>::value && NI >= 5) ? 3 : 1;
#pragma unroll UQ
        for (int q3 = 0; q3 < NQ; ++q3) {
            RC d[9];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const RC *s2c = s2 + c * 3 * O2 + col;
                RC r0 = 0, r1 = 0, r2 = 0;
#pragma unroll
                for (int i3 = 0; i3 < NI; ++i3) {
                    const RC Bq = B[q3 * NI + i3], Gq = G[q3 * NI + i3];
                    acc_add(r0, Bq * s2c[i3 * NQ * NQ]);
                    acc_add(r1, Bq * s2c[O2 + i3 * NQ * NQ]);
                    acc_add(r2, Gq * s2c[2 * O2 + i3 * NQ * NQ]);
                }
                d[c * 3 + 0] = norm(r0);
                d[c * 3 + 1] = norm(r1);
                d[c * 3 + 2] = norm(r2);
            }
            RC y[9];
#pragma unroll
            for (int r = 0; r < 9; ++r) y[r] = 0;
#pragma unroll
            for (int r = 0; r < 9; ++r)
#pragma unroll
                for (int s = r; s < 9; ++s) {
                    const RC h = C::PAIRS ? He[C::hoff(pidx<9>(r, s), q3 * NQ * NQ + col)]
                                          : Hc[pidx<9>(r, s) * NQD + q3 * NQ * NQ];
                    acc_add(y[r], h * d[s]);
                    if (s != r) acc_add(y[s], h * d[r]);
                }
#pragma unroll
            for (int r = 0; r < 9; ++r) {
                const RC yr = norm(y[r]);
#pragma unroll
                for (int i3 = 0; i3 < NI; ++i3)
                    acc_add(z[r][i3], ((r % 3) == 2 ? G[q3 * NI + i3] : B[q3 * NI + i3]) * yr);
            }
        }
        // the thread's own (q1, q2) entries of the stage values: overwrite in place
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                RC *s2c = s2 + c * 3 * O2 + i3 * NQ * NQ + col;
                s2c[0] = norm(z[c * 3 + 0][i3]);
                s2c[O2] = norm(z[c * 3 + 1][i3]);
                s2c[2 * O2] = norm(z[c * 3 + 2][i3]);
            }
    }
    __syncthreads();

    // ---- transposed stages 2 and 3 per component
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        const RC *s2c = s2 + c * 3 * O2;
        if (valid && tx < NQ && ty < NI) {
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                RC a = 0, b = 0;
#pragma unroll
                for (int q2 = 0; q2 < NQ; ++q2) {
                    const RC Bq = B[q2 * NI + ty], Gq = G[q2 * NI + ty];
                    acc_add(a, Bq * s2c[(i3 * NQ + q2) * NQ + tx]);
                    acc_add(b, Gq * s2c[O2 + (i3 * NQ + q2) * NQ + tx]);
                    acc_add(b, Bq * s2c[2 * O2 + (i3 * NQ + q2) * NQ + tx]);
                }
                s1[(i3 * NI + ty) * NQ + tx] = norm(a);
                s1[O1 + (i3 * NI + ty) * NQ + tx] = norm(b);
            }
        }
        __syncthreads();
        if (valid && tx < NI && ty < NI) {
            RV *o_e = ev + (int64_t)c * P.E * NP + e * NP;
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                RC o = 0;
#pragma unroll
                for (int q1 = 0; q1 < NQ; ++q1) {
                    acc_add(o, G[q1 * NI + tx] * s1[(i3 * NI + ty) * NQ + q1]);
                    acc_add(o, B[q1 * NI + tx] * s1[O1 + (i3 * NI + ty) * NQ + q1]);
                }
                ev_store(&o_e[(i3 * NI + ty) * NI + tx], norm(o));
            }
        }
        __syncthreads();      // s1 is reused by the next component
    }
}

}  // namespace tmop
