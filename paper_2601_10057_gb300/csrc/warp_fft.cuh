// warp_fft.cuh -- warp-level four-step FFT of whole grid lines (FP32 path).
//
// A line of M = E * G complex values is held by a group of G lanes, E values
// per lane (lane n2 holds z[G n1 + n2], n1 = 0..E-1):
//   1. E-point DFT over n1 in registers (radix-2 decimation in frequency,
//      exact compile-time twiddles; output in bit-reversed register order);
//   2. twiddle by W_M^{n2 k1} (table tw2[k1][n2], coalesced across lanes);
//   3. transpose through the line's shared-memory buffer (rows padded to
//      G + 1 values, or unpadded and XOR-swizzled; both conflict-free);
//   4. E/G G-point DFTs over n2 in registers; the result Z[k1 + E k2] is
//      written to the buffer in natural order.
// One smem round trip per stage pair instead of one per radix-8 stage, no
// block barriers (only __syncwarp), and 32 independent values per lane.
// Supported lines: M in {64, ..., 4096} (N = 2M in 128 .. 8192); the shapes
// E x G are listed below (Shape).  A group of G = 32 W lanes (W = 2, 4)
// spans W warps: its lanes synchronise through a named barrier of the line
// (id 1 + line slot, G threads) instead of __syncwarp.  Shapes with E < G
// take fourstep_split for steps 3-4.
#pragma once
#include <type_traits>
#include "dct_device.cuh"

namespace ccm {
namespace wf {

__device__ __forceinline__ void w32(int j, double& c, double& s) {
    switch (j & 31) {
        case 0: c = 1.0; s = 0.0; break;
        case 1: c = 0.9807852804032304; s = 0.19509032201612825; break;
        case 2: c = 0.9238795325112867; s = 0.3826834323650898; break;
        case 3: c = 0.8314696123025452; s = 0.5555702330196022; break;
        case 4: c = 0.7071067811865476; s = 0.7071067811865475; break;
        case 5: c = 0.5555702330196023; s = 0.8314696123025452; break;
        case 6: c = 0.38268343236508984; s = 0.9238795325112867; break;
        case 7: c = 0.19509032201612833; s = 0.9807852804032304; break;
        case 8: c = 0.0; s = 1.0; break;
        case 9: c = -0.1950903220161282; s = 0.9807852804032304; break;
        case 10: c = -0.3826834323650897; s = 0.9238795325112867; break;
        case 11: c = -0.555570233019602; s = 0.8314696123025455; break;
        case 12: c = -0.7071067811865475; s = 0.7071067811865476; break;
        case 13: c = -0.8314696123025453; s = 0.5555702330196022; break;
        case 14: c = -0.9238795325112867; s = 0.3826834323650899; break;
        case 15: c = -0.9807852804032304; s = 0.1950903220161286; break;
        case 16: c = -1.0; s = 0.0; break;
        case 17: c = -0.9807852804032304; s = -0.19509032201612836; break;
        case 18: c = -0.9238795325112868; s = -0.38268343236508967; break;
        case 19: c = -0.8314696123025455; s = -0.555570233019602; break;
        case 20: c = -0.7071067811865477; s = -0.7071067811865475; break;
        case 21: c = -0.5555702330196022; s = -0.8314696123025452; break;
        case 22: c = -0.38268343236509034; s = -0.9238795325112865; break;
        case 23: c = -0.19509032201612866; s = -0.9807852804032303; break;
        case 24: c = 0.0; s = -1.0; break;
        case 25: c = 0.1950903220161283; s = -0.9807852804032304; break;
        case 26: c = 0.38268343236509; s = -0.9238795325112866; break;
        case 27: c = 0.5555702330196018; s = -0.8314696123025455; break;
        case 28: c = 0.7071067811865474; s = -0.7071067811865477; break;
        case 29: c = 0.8314696123025452; s = -0.5555702330196022; break;
        case 30: c = 0.9238795325112865; s = -0.3826834323650904; break;
        case 31: c = 0.9807852804032303; s = -0.19509032201612872; break;
        default: c = 1.0; s = 0.0; break;
    }
}

// 64th roots of unity: w64(j) = cos(2 pi j / 64), sin(2 pi j / 64), j = 0..63
__device__ __forceinline__ void w64(int j, double& c, double& s) {
    switch (j & 63) {
        case 0: c = 1.0; s = 0.0; break;
        case 1: c = 0.9951847266721969; s = 0.0980171403295606; break;
        case 2: c = 0.9807852804032304; s = 0.19509032201612825; break;
        case 3: c = 0.9569403357322088; s = 0.29028467725446233; break;
        case 4: c = 0.9238795325112867; s = 0.3826834323650898; break;
        case 5: c = 0.881921264348355; s = 0.47139673682599764; break;
        case 6: c = 0.8314696123025452; s = 0.5555702330196022; break;
        case 7: c = 0.773010453362737; s = 0.6343932841636455; break;
        case 8: c = 0.7071067811865476; s = 0.7071067811865475; break;
        case 9: c = 0.6343932841636455; s = 0.773010453362737; break;
        case 10: c = 0.5555702330196023; s = 0.8314696123025452; break;
        case 11: c = 0.4713967368259978; s = 0.8819212643483549; break;
        case 12: c = 0.38268343236508984; s = 0.9238795325112867; break;
        case 13: c = 0.29028467725446233; s = 0.9569403357322089; break;
        case 14: c = 0.19509032201612833; s = 0.9807852804032304; break;
        case 15: c = 0.09801714032956077; s = 0.9951847266721968; break;
        case 16: c = 0.0; s = 1.0; break;
        case 17: c = -0.09801714032956065; s = 0.9951847266721969; break;
        case 18: c = -0.1950903220161282; s = 0.9807852804032304; break;
        case 19: c = -0.29028467725446216; s = 0.9569403357322089; break;
        case 20: c = -0.3826834323650897; s = 0.9238795325112867; break;
        case 21: c = -0.4713967368259977; s = 0.881921264348355; break;
        case 22: c = -0.555570233019602; s = 0.8314696123025455; break;
        case 23: c = -0.6343932841636454; s = 0.7730104533627371; break;
        case 24: c = -0.7071067811865475; s = 0.7071067811865476; break;
        case 25: c = -0.773010453362737; s = 0.6343932841636455; break;
        case 26: c = -0.8314696123025453; s = 0.5555702330196022; break;
        case 27: c = -0.8819212643483549; s = 0.47139673682599786; break;
        case 28: c = -0.9238795325112867; s = 0.3826834323650899; break;
        case 29: c = -0.9569403357322088; s = 0.2902846772544624; break;
        case 30: c = -0.9807852804032304; s = 0.1950903220161286; break;
        case 31: c = -0.9951847266721968; s = 0.09801714032956083; break;
        case 32: c = -1.0; s = 0.0; break;
        case 33: c = -0.9951847266721969; s = -0.09801714032956059; break;
        case 34: c = -0.9807852804032304; s = -0.19509032201612836; break;
        case 35: c = -0.9569403357322089; s = -0.2902846772544621; break;
        case 36: c = -0.9238795325112868; s = -0.38268343236508967; break;
        case 37: c = -0.881921264348355; s = -0.47139673682599764; break;
        case 38: c = -0.8314696123025455; s = -0.555570233019602; break;
        case 39: c = -0.7730104533627371; s = -0.6343932841636453; break;
        case 40: c = -0.7071067811865477; s = -0.7071067811865475; break;
        case 41: c = -0.6343932841636459; s = -0.7730104533627367; break;
        case 42: c = -0.5555702330196022; s = -0.8314696123025452; break;
        case 43: c = -0.47139673682599786; s = -0.8819212643483549; break;
        case 44: c = -0.38268343236509034; s = -0.9238795325112865; break;
        case 45: c = -0.29028467725446244; s = -0.9569403357322088; break;
        case 46: c = -0.19509032201612866; s = -0.9807852804032303; break;
        case 47: c = -0.09801714032956045; s = -0.9951847266721969; break;
        case 48: c = 0.0; s = -1.0; break;
        case 49: c = 0.09801714032956009; s = -0.9951847266721969; break;
        case 50: c = 0.1950903220161283; s = -0.9807852804032304; break;
        case 51: c = 0.29028467725446205; s = -0.9569403357322089; break;
        case 52: c = 0.38268343236509; s = -0.9238795325112866; break;
        case 53: c = 0.4713967368259976; s = -0.881921264348355; break;
        case 54: c = 0.5555702330196018; s = -0.8314696123025455; break;
        case 55: c = 0.6343932841636456; s = -0.7730104533627369; break;
        case 56: c = 0.7071067811865474; s = -0.7071067811865477; break;
        case 57: c = 0.7730104533627367; s = -0.6343932841636459; break;
        case 58: c = 0.8314696123025452; s = -0.5555702330196022; break;
        case 59: c = 0.8819212643483548; s = -0.4713967368259979; break;
        case 60: c = 0.9238795325112865; s = -0.3826834323650904; break;
        case 61: c = 0.9569403357322088; s = -0.2902846772544625; break;
        case 62: c = 0.9807852804032303; s = -0.19509032201612872; break;
        case 63: c = 0.9951847266721969; s = -0.0980171403295605; break;
        default: c = 1.0; s = 0.0; break;
    }
}

// x * W_R^i (forward: exp(-2 pi i I / R); INV: conjugate)
template <typename T, int R, bool INV>
__device__ __forceinline__ cplx<T> twid(cplx<T> x, int i) {
    constexpr int RM = R > 32 ? 64 : 32;          // table of RM-th roots of unity
    const int j = (i * (RM / R)) & (RM - 1);
    if (j == 0) return x;
    if (j == RM / 4) return INV ? mk(-x.y, x.x) : mk(x.y, -x.x);
    if (j == RM / 2) return mk(-x.x, -x.y);
    if (j == 3 * RM / 4) return INV ? mk(x.y, -x.x) : mk(-x.y, x.x);
    double c, s;
    if (RM == 64) w64(j, c, s); else w32(j, c, s);
    const T cc = (T)c, ss = INV ? (T)s : (T)(-s);     // W = c + i ss
    return mk(x.x * cc - x.y * ss, x.x * ss + x.y * cc);
}

// In-register radix-2 DIF on v[OFF .. OFF + R): natural input, output
// v[OFF + r] = X[bitrev_R(r)].
template <typename T, int R, bool INV, int OFF>
struct DIF {
    static __device__ __forceinline__ void run(cplx<T>* v) {
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            const cplx<T> a = v[OFF + i], b = v[OFF + i + R / 2];
            v[OFF + i] = a + b;
            v[OFF + i + R / 2] = twid<T, R, INV>(a - b, i);
        }
        DIF<T, R / 2, INV, OFF>::run(v);
        DIF<T, R / 2, INV, OFF + R / 2>::run(v);
    }
};
template <typename T, bool INV, int OFF>
struct DIF<T, 1, INV, OFF> {
    static __device__ __forceinline__ void run(cplx<T>*) {}
};

template <int R> __host__ __device__ constexpr int bitrev(int r) {
    int o = 0;
    for (int b = 1, q = R >> 1; b < R; b <<= 1, q >>= 1)
        if (r & b) o |= q;
    return o;
}

// Line shapes M = E x G (E values on each of G lanes).  S selects a variant:
// the forward transforms run 2048-point lines as 64 x 32 (one warp per line)
// and 4096-point lines as 64 x 64; the inverse kernels, which wait on memory
// and gain from the lower register use, take 32 x 64 and 32 x 128 (two and
// four warps per line, fourstep_split).
template <int M> struct ShapeBase;
template <> struct ShapeBase<64>   { static constexpr int E = 8,  G = 8;  };
template <> struct ShapeBase<128>  { static constexpr int E = 16, G = 8;  };
template <> struct ShapeBase<256>  { static constexpr int E = 16, G = 16; };
template <> struct ShapeBase<512>  { static constexpr int E = 32, G = 16; };
template <> struct ShapeBase<1024> { static constexpr int E = 32, G = 32; };
template <> struct ShapeBase<2048> { static constexpr int E = 64, G = 32; };
template <> struct ShapeBase<4096> { static constexpr int E = 64, G = 64; };
template <int M, int S = 0> struct Shape : ShapeBase<M> {};
template <> struct Shape<2048, 1> { static constexpr int E = 32, G = 64; };
template <> struct Shape<4096, 1> { static constexpr int E = 32, G = 128; };

// Lane n2 of its line's group and the line's slot in the CTA: G <= 32 puts
// 32 / G lines in a warp; G = 64, 128 spreads a line over 2, 4 consecutive
// warps.
template <int M, int S = 0> __device__ __forceinline__ void lane_geo(int& n2, int& slot) {
    constexpr int G = Shape<M, S>::G;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if constexpr (G <= 32) {
        n2 = lane % G;
        slot = warp * (32 / G) + lane / G;
    } else {
        n2 = lane + 32 * (warp % (G / 32));
        slot = warp / (G / 32);
    }
}

// Barrier of one line's lane group: the warp's own lanes for G <= 32, the
// warps of the line (named barrier 1 + slot; every one of their G threads
// arrives) for G = 64, 128.
template <int G> __device__ __forceinline__ void line_sync(int slot) {
    if constexpr (G <= 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" :: "r"(1 + slot), "r"(G) : "memory");
    }
}

// Per-line buffer length (complex values) for the transpose and the
// natural-order result.  Padded (SWZ = false): rows of G + 1 values; + 2 so
// that, as float rows, consecutive line buffers sit 4 banks apart (the
// strided reads of the transposed writes).  Swizzled (SWZ = true): M values
// + 2, for kernels that need more lines per SM.
template <int M, bool SWZ = false, int S = 0> __host__ __device__ constexpr int buf_len() {
    return Shape<M, S>::E < Shape<M, S>::G                                          // fourstep_split's rows
             ? Shape<M, S>::E * (Shape<M, S>::G + Shape<M, S>::G / Shape<M, S>::E)
         : SWZ ? M + 2 : Shape<M, S>::E * (Shape<M, S>::G + 1) + 2;
}

// Position of element c of transpose row R (E rows of G values).  Padded:
// R (G + 1) + c.  Swizzled: R G + (c ^ swz(R)) with J = E / G and, for
// E <= 32, swz(R) = 2 (R / J) mod G: the writes (one row, all lanes of a
// group) touch distinct banks within each half-warp, and since swz is even
// the columns 2p, 2p + 1 stay adjacent and in order, so a lane reads two
// values of its row (n2 J + j) with one 16-byte load, on distinct banks within
// each quarter-warp for G >= 16.  For E = 64, swz(R) = (R / J) mod G with
// 8-byte reads (measured faster there).
template <int M, int S = 0> __host__ __device__ constexpr bool wide_reads() { return Shape<M, S>::E <= 32; }
template <int M, bool SWZ, int S = 0> __device__ __forceinline__ int tpos(int R, int c) {
    constexpr int G = Shape<M, S>::G, J = Shape<M, S>::E / Shape<M, S>::G, W = wide_reads<M, S>() ? 2 : 1;
    return SWZ ? R * G + (c ^ ((W * (R / J)) & (G - 1))) : R * (G + 1) + c;
}

// The four steps for lines of G = R E lanes (E values each, R = 2 or 4): the
// E-point DFTs and the twiddles as below, then each G-point row k1 of the
// transpose is split over R adjacent lanes (lane R k1 + q takes the columns
// R t + q, t = 0 .. E-1), each lane takes an E-point DFT Y_q of its part,
// multiplies it by W_G^{q k} (U_q), and the R lanes combine by an R-point DFT
// through shuffles:
//   X[k1 + E (k + E s)] = sum_q W_R^{q s} U_q[k]        (conjugates for INV),
// R = 2 in one radix-2 step (lane q keeps s = q), R = 4 in two (pairs q, q^2,
// then q, q^1; lane q keeps s = bit-reversed q).  W_G^{q k} = W_M^{E q k} is
// the table entry of k1 = k, n2 = E q: tw2[k G + E q].  Transpose rows are
// padded to G + R values:
// the row writes (one row, all lanes) and the part-row reads (16 / R rows and
// all R parts per half-warp, 8-byte words) touch distinct banks.
template <typename T, int M, bool INV, int S = 0>
__device__ __forceinline__ void fourstep_split(cplx<T>* v, cplx<T>* buf, const cplx<T>* __restrict__ tw2, int n2, int slot) {
    constexpr int E = Shape<M, S>::E, G = Shape<M, S>::G, R = G / E, P = G + R;
    static_assert(R == 2 || R == 4, "two or four lanes per transpose row");
    DIF<T, E, INV, 0>::run(v);                   // v[r] = X1[k1 = bitrev(r)] of column n2
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int k1 = bitrev<E>(r);
        const cplx<T> w = tw2[k1 * G + n2];
        buf[k1 * P + n2] = INV ? cmulc(v[r], w) : cmul(v[r], w);
    }
    line_sync<G>(slot);
    const int k1 = n2 / R, q = n2 % R;
#pragma unroll
    for (int t = 0; t < E; ++t) v[t] = buf[k1 * P + R * t + q];
    line_sync<G>(slot);
    DIF<T, E, INV, 0>::run(v);                   // v[r] = Y_q[k = bitrev(r)]
    constexpr unsigned FULL = 0xffffffffu;
    if constexpr (R == 2) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int k = bitrev<E>(r);
            const T px = __shfl_xor_sync(FULL, v[r].x, 1);
            const T py = __shfl_xor_sync(FULL, v[r].y, 1);
            const cplx<T> y0 = q ? mk(px, py) : v[r];
            const cplx<T> y1 = twid<T, G, INV>(q ? v[r] : mk(px, py), k);
            buf[k1 + E * (k + E * q)] = q ? y0 - y1 : y0 + y1;
        }
    } else {
        const int s = ((q & 1) << 1) | (q >> 1);  // output index of this lane
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int k = bitrev<E>(r);
            const cplx<T> w = tw2[k * G + E * q];            // W_G^{q k}
            cplx<T> u = INV ? cmulc(v[r], w) : cmul(v[r], w);
            // pairs (q, q ^ 2): lanes q < 2 keep U_q + U_{q^2}, lanes q >= 2 keep U_{q^2} - U_q
            T px = __shfl_xor_sync(FULL, u.x, 2), py = __shfl_xor_sync(FULL, u.y, 2);
            u = (q & 2) ? mk(px - u.x, py - u.y) : mk(u.x + px, u.y + py);
            // pairs (q, q ^ 1): even lanes X = A_q + w4 A_{q^1}, odd lanes X = A_{q^1} - w4 A_q,
            // w4 = 1 for q < 2 and W_4 (-i; +i for INV) for q >= 2
            px = __shfl_xor_sync(FULL, u.x, 1); py = __shfl_xor_sync(FULL, u.y, 1);
            const cplx<T> a = (q & 1) ? mk(px, py) : u, b = (q & 1) ? u : mk(px, py);
            const cplx<T> wb = (q & 2) ? (INV ? mk(-b.y, b.x) : mk(b.y, -b.x)) : b;
            buf[k1 + E * (k + E * s)] = (q & 1) ? a - wb : a + wb;
        }
    }
    line_sync<G>(slot);
}

// Steps 1-4.  v: this lane's E values in four-step order.  buf: this line's
// buffer.  On return buf[k] = Z[k], k = 0..M-1 (visible to the warp).
template <typename T, int M, bool INV, bool SWZ = false, int S = 0>
__device__ __forceinline__ void fourstep(cplx<T>* v, cplx<T>* buf, const cplx<T>* __restrict__ tw2, int n2, int slot) {
  if constexpr (Shape<M, S>::E < Shape<M, S>::G) {
    fourstep_split<T, M, INV, S>(v, buf, tw2, n2, slot);
  } else {
    constexpr int E = Shape<M, S>::E, G = Shape<M, S>::G, J = E / G;
    DIF<T, E, INV, 0>::run(v);
    if constexpr (!INV) {
        // twiddles W_M^{n2 k1}: k1 = bitrev(r) is below E/2 for even r; for odd
        // r it is the even partner's + E/2, so W^{n2 k1} = W^{n2 k1'} W^{(E/2) n2}
        // (half the table loads; measured faster in the forward kernels, which
        // are shared-memory/load bound, slower in the inverse ones)
        const cplx<T> wh = tw2[(E / 2) * G + n2];
#pragma unroll
        for (int r = 0; r < E; r += 2) {
            const int k1 = bitrev<E>(r);
            const cplx<T> w = tw2[k1 * G + n2];
            buf[tpos<M, SWZ, S>(k1, n2)] = cmul(v[r], w);
            buf[tpos<M, SWZ, S>(k1 + E / 2, n2)] = cmul(v[r + 1], cmul(w, wh));
        }
    } else {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int k1 = bitrev<E>(r);
            buf[tpos<M, SWZ, S>(k1, n2)] = cmulc(v[r], tw2[k1 * G + n2]);
        }
    }
    line_sync<G>(slot);
    if constexpr (SWZ && wide_reads<M, S>() && std::is_same<T, float>::value) {
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
            for (int m = 0; m < G; m += 2) {
                const float4 q = *reinterpret_cast<const float4*>(buf + tpos<M, SWZ, S>(n2 * J + j, m));
                v[j * G + m] = mk(q.x, q.y);
                v[j * G + m + 1] = mk(q.z, q.w);
            }
    } else {
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
            for (int m = 0; m < G; ++m) v[j * G + m] = buf[tpos<M, SWZ, S>(n2 * J + j, m)];
    }
    line_sync<G>(slot);
#pragma unroll
    for (int j = 0; j < J; ++j) {
        if (j == 0) DIF<T, G, INV, 0>::run(v);
        else DIF<T, G, INV, G>::run(v);
    }
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
        for (int r = 0; r < G; ++r) buf[(n2 * J + j) + E * bitrev<G>(r)] = v[j * G + r];
    line_sync<G>(slot);
  }
}

// Forward pack from a real line x in global memory (16-byte aligned):
// z[m] = (x[4m], x[4m+2]), z[M-1-m] = (x[4m+3], x[4m+1]); lane n2 needs
// z[G n1 + n2]; the mirrored half comes from lane n2 ^ (G-1).
template <int M>
__device__ __forceinline__ void pack_fwd_global(const float* __restrict__ x, cplx<float>* v, int n2) {
    constexpr int E = Shape<M>::E, G = Shape<M>::G;
#pragma unroll
    for (int n1 = 0; n1 < E / 2; ++n1) {
        const float4 q = __ldcg(reinterpret_cast<const float4*>(x) + (G * n1 + n2));   // L2 only: keeps L1 for the tables
        v[n1] = mk(q.x, q.z);
        if constexpr (G <= 32) {
            const float ox = __shfl_xor_sync(0xffffffffu, q.w, G - 1);
            const float oy = __shfl_xor_sync(0xffffffffu, q.y, G - 1);
            v[E - 1 - n1] = mk(ox, oy);
        } else {
            // the partner lane G - 1 - n2 sits in the other warp: load its quad too
            const float4 p = __ldg(reinterpret_cast<const float4*>(x) + (G * n1 + (G - 1 - n2)));
            v[E - 1 - n1] = mk(p.w, p.y);
        }
    }
}

// Twiddles of the pair (k, M-k) for the lean post-/pre-processing below
// (host-computed in FP64 from the closed forms; the 1/2 of the even/odd
// split, the DCT normalisation and the e^{-+i pi/4} rotation are folded in):
//   wn = e^{-2 pi i k / N};
//   forward: a = c_k / 2 e^{-i pi k / (2N)} (c_0 = sqrt(1/N), c_k = sqrt(2/N)),
//            b = sqrt(2/N) / 2 e^{-i pi/4} e^{+i pi k / (2N)};
//   inverse: a = s_k / 2 e^{+i pi k / (2N)} (s_0 = 1/(M sqrt(1/N)), s_k = 1/(M sqrt(2/N))),
//            b = s_k' / 2 e^{+i pi/4} e^{-i pi k / (2N)} (s_k' = 1/(M sqrt(2/N))).
struct PairTw { float wnx, wny, ax, ay, bx, by; };

// Device table of the pairs k = 0 .. NP-1: one float4 (wnx, wny, ax, ay)
// per pair (lanes reading consecutive pairs read contiguous 16-byte words).
// b follows from a for k >= 1, where both carry the same factor
// sqrt(2/N)/2 (forward) or 1/(M sqrt(2/N))/2 (inverse):
//   forward b = e^{-i pi/4} conj(a),  inverse b = e^{+i pi/4} conj(a);
// b of the pair k = 0 (where a has the k = 0 factor) is stored as b0.
struct PairTwTab { const float4* __restrict__ wa; float2 b0; };

template <bool INV>
__device__ __forceinline__ PairTw load_pair_tw(const PairTwTab& t, int k) {
    const float4 u = __ldg(t.wa + k);
    constexpr float h = 0.70710678118654752440f;
    float bx = INV ? (u.z + u.w) * h : (u.z - u.w) * h;
    float by = INV ? (u.z - u.w) * h : -(u.z + u.w) * h;
    if (k == 0) { bx = t.b0.x; by = t.b0.y; }
    return PairTw{u.x, u.y, u.z, u.w, bx, by};
}

// Forward post-process of the pair (k, M-k): A = Z[k], B = Z[M-k].  With
// P = A + conj B, Q = A - conj B and U = wn Q, the half-length spectrum gives
// V[k] ~ P - iU and V[M-k] ~ conj(P + iU), so
//   X[k] = Re(a S), X[N-k] = -Im(a S), S = P - iU;
//   X[M-k] = Re(b R), X[M+k] = -Im(b R), R = conj(P + iU).
__device__ __forceinline__ Quad<float> post_pair_lean(cplx<float> A, cplx<float> B, const PairTw& t) {
    const float Px = A.x + B.x, Py = A.y - B.y, Qx = A.x - B.x, Qy = A.y + B.y;
    const float Ux = t.wnx * Qx - t.wny * Qy, Uy = t.wnx * Qy + t.wny * Qx;
    const float Sx = Px + Uy, Sy = Py - Ux;
    const float Rx = Px - Uy, Ry = -(Py + Ux);
    Quad<float> q;
    q.xk = t.ax * Sx - t.ay * Sy;
    q.xNk = -(t.ax * Sy + t.ay * Sx);
    q.xMk = t.bx * Rx - t.by * Ry;
    q.xMpk = -(t.bx * Ry + t.by * Rx);
    return q;
}

// Inverse pre-process of the pair (k, M-k) from X[k], X[N-k] (0 for k = 0),
// X[M-k], X[M+k]: Vk = a (X[k] - i X[N-k]), Vm = b (X[M-k] - i X[M+k]),
// s = Vk + conj Vm, d = Vk - conj Vm, tt = d conj(wn); then
// z[k] = s + i tt and z[M-k] = conj(s) + i conj(tt).
__device__ __forceinline__ void pre_pair_lean(const Quad<float>& X, const PairTw& t, cplx<float>& zk, cplx<float>& zMk) {
    const float Vkx = t.ax * X.xk + t.ay * X.xNk, Vky = t.ay * X.xk - t.ax * X.xNk;
    const float Vmx = t.bx * X.xMk + t.by * X.xMpk, Vmy = t.by * X.xMk - t.bx * X.xMpk;
    const float sx = Vkx + Vmx, sy = Vky - Vmy, dx = Vkx - Vmx, dy = Vky + Vmy;
    const float tx = dx * t.wnx + dy * t.wny, ty = dy * t.wnx - dx * t.wny;
    zk = mk(sx - ty, sy + tx);
    zMk = mk(sx + ty, tx - sy);
}

// Forward post-process of the pair (k, M-k) from natural-order Z values.
template <typename T>
__device__ __forceinline__ Quad<T> post_pair(cplx<T> A, cplx<T> B, int k, PostTw<T> tw, T cn0, T cn) {
    const T h = (T)0.70710678118654752440;
    cplx<T> WN = mk(tw.cN, -tw.sN), W4 = mk(tw.c4, -tw.s4);
    cplx<T> E = scale(A + conj_(B), (T)0.5);
    cplx<T> D = scale(A - conj_(B), (T)0.5);
    cplx<T> O = mk(D.y, -D.x);
    cplx<T> W = cmul(W4, E + cmul(WN, O));
    cplx<T> Dc = conj_(D);
    cplx<T> O2 = mk(-Dc.y, Dc.x);
    cplx<T> WN2 = mk(-WN.x, WN.y);
    cplx<T> W4c = conj_(W4);
    cplx<T> W42 = mk(h * (W4c.x + W4c.y), h * (W4c.y - W4c.x));
    cplx<T> W2 = cmul(W42, conj_(E) + cmul(WN2, O2));
    Quad<T> q;
    q.xk = (k == 0 ? cn0 : cn) * W.x;
    q.xNk = -cn * W.y;
    q.xMk = cn * W2.x;
    q.xMpk = -cn * W2.y;
    return q;
}

}  // namespace wf
}  // namespace ccm
