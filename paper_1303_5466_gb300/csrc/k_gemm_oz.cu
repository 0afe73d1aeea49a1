// k_gemm_oz.cu -- FP64 grouped GEMM from exact products of 7-bit digit slices on the bf16 tensor
// cores: the E products of Algorithm 1 (W = Phi_{:,r} T^T + Phi_{:,s}, E^{-1} = T W_r + W_s), the
// rank-64 updates of the blocked sweep (k_sweep_bl.cu) and of the blocked T = R11^{-1} R12
// (k_idt_bl.cu).
//
// This GPU runs FP64 FMAs at 1.2 TFLOP/s and bf16 tensor-core products (mma.sync, FP32
// accumulation) at 0.6 PFLOP/s.  Each FP64 entry is written as a sum of eight signed 7-bit
// digits against a power of two shared by its row of A (or column of B): x = sum_s q_s 2^(E-7-7s),
// |q_s| <= 127, exact up to the 56th bit below the row's largest entry.  A digit is an integer
// that bf16 holds exactly, and so is the product of two; a K-chunk of 128 of them, summed over
// the at most 8 digit pairs (i, j) of one level l = i + j, stays below 2^24 and is therefore exact
// in the tensor core's FP32 accumulator.  The eight level sums of a chunk are combined in int64
// (W_A = sum_{l<4} S_l 2^(7(3-l)), W_B the same for l = 4..7) and summed over the chunks exactly,
// so C = 2^(EA+EB-35) (W_A + 2^-28 W_B) carries one rounding, against K roundings of a chain of
// FP64 FMAs.  Levels above 7 (products below 2^-56 of the row and column maxima) are left out:
// the result differs from the exact product by at most about K 2^-56 max|A_i,:| max|B_:,j|.
//
// Launch: one warp per row of A and per column of B finds its exponent and writes the line's
// digits (slice-major bf16, K padded to 32); then one CTA of 8 warps per 64 x 32 tile of C, the
// warps 16 x 16 each (two m16n8k16 tiles), K in stages of 16 digits that cp.async copies into
// one of two shared-memory buffers while the previous stage's products run.
#include <algorithm>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>

#include "k_common.cuh"

namespace rs {

namespace {

constexpr int OZ_BM = 64, OZ_BN = 32, OZ_BK = 16, OZ_NT = 256;
constexpr int OZ_S = 8;               // digit slices per entry
constexpr int OZ_CHUNK = 128;         // K per exact FP32 level sum
constexpr int OZ_KP = 32;             // a digit line's K, padded to a multiple of this
constexpr int OZ_LD = OZ_BK + 8;      // padded row of a slice tile (bf16): 48 B, conflict-free fragments
constexpr int OZ_BUF = OZ_S * (OZ_BM + OZ_BN) * OZ_LD;   // bf16 of one stage buffer

__host__ __device__ inline int oz_kp(int K) { return (K + OZ_KP - 1) / OZ_KP * OZ_KP; }

__device__ __forceinline__ double oz_a(const GemmProb& P, const double* A, int i, int k)
{
    return P.ta ? A[(int64_t)i * P.lda + k] : A[(int64_t)k * P.lda + i];
}
__device__ __forceinline__ double oz_b(const GemmProb& P, const double* B, int k, int j)
{
    return P.tb ? B[(int64_t)k * P.ldb + j] : B[(int64_t)j * P.ldb + k];
}

// |x| 2^(56-E) truncated to an integer Z < 2^56 (|x| < 2^E), and the sign of x.
__device__ __forceinline__ unsigned long long oz_fixed(double x, int E, bool& neg)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int ef = (int)((u >> 52) & 0x7ff);
    unsigned long long Z = 0;
    if (ef != 0) {                                   // zeros and subnormals: no digits
        const unsigned long long mt = (u & ((1ull << 52) - 1)) | (1ull << 52);
        const int sh = (ef - 1023) + 4 - E;          // |x| < 2^E, so sh <= 3
        if (sh >= 0) Z = mt << sh;
        else if (sh > -64) Z = mt >> (-sh);
    }
    neg = (u >> 63) != 0;
    return Z;
}

// bf16 bits of the signed digit s of Z (bits 49-7s .. 55-7s): the 7-bit integer through an FP32
// add of a power of two (exact), the top half of its bits, and the sign bit.
__device__ __forceinline__ uint32_t oz_digit(unsigned long long Z, bool neg, int s)
{
    const uint32_t d = (uint32_t)(Z >> (49 - 7 * s)) & 127u;
    const float f = __uint_as_float(0x4B000000u | d) - 8388608.0f;
    return (__float_as_uint(f) >> 16) | (neg ? 0x8000u : 0u);
}

// Digits of two entries (consecutive in k) of one row, one 32-bit word per slice.
__device__ __forceinline__ void oz_split2(double x0, double x1, int E, uint32_t* out, int stride_words)
{
    bool n0, n1;
    const unsigned long long Z0 = oz_fixed(x0, E, n0), Z1 = oz_fixed(x1, E, n1);
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) out[s * stride_words] = oz_digit(Z0, n0, s) | (oz_digit(Z1, n1, s) << 16);
}

// (wa 2^28 + wb) 2^e2, rounded to nearest (ties to even) once, in integer operations.
__device__ __forceinline__ double oz_round(long long wa, long long wb, int e2)
{
    const __int128 T = (__int128)wa * ((__int128)1 << 28) + (__int128)wb;
    const bool neg = T < 0;
    const unsigned __int128 M = neg ? (unsigned __int128)(-T) : (unsigned __int128)T;
    if (M == 0) return 0.0;
    const unsigned long long hi = (unsigned long long)(M >> 64), lo = (unsigned long long)M;
    int sh = (hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo)) - 53;
    unsigned long long q;
    if (sh > 0) {
        q = (unsigned long long)(M >> sh);
        const unsigned __int128 rem = M - ((unsigned __int128)q << sh);
        const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
        if (rem > half || (rem == half && (q & 1ull))) {
            if (++q == (1ull << 53)) {
                q >>= 1;
                ++sh;
            }
        }
    } else {
        q = (unsigned long long)M << (-sh);
    }
    const int ef = sh + e2 + 1075;                   // value = q 2^(sh + e2), 2^52 <= q < 2^53
    if (ef <= 0 || ef >= 2047) return ldexp(fma((double)wb, 0x1p-28, (double)wa), e2 + 28);
    return __longlong_as_double((long long)(((unsigned long long)neg << 63) | ((unsigned long long)ef << 52) |
                                            (q & ((1ull << 52) - 1))));
}

__device__ __forceinline__ void oz_mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One warp per line (a row of A or a column of B): its exponent E (max |x| < 2^E, 0 for an
// all-zero line; in integer operations, this GPU's FP64 pipe being its scarcest), then the
// digits of its K entries (zero up to the padded length), slice-major: line base + s Kp + k.
// eoff[p] is problem p's first line, eoff[np + 1 + p] its first digit.
__global__ void __launch_bounds__(256) oz_split_kernel(const GemmProb* __restrict__ probs, int np,
        const int64_t* __restrict__ eoff, int64_t nlines, const double* __restrict__ Ab,
        const double* __restrict__ Bb, int* __restrict__ ex, __nv_bfloat16* __restrict__ dig)
{
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nlines) return;
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (eoff[mid] <= w) lo = mid; else hi = mid - 1;
    }
    const GemmProb P = probs[lo];
    const int idx = (int)(w - eoff[lo]);
    const bool isA = idx < P.M;
    const double* A = Ab + P.a_off;
    const double* B = Bb + P.b_off;
    auto val = [&](int k) { return isA ? oz_a(P, A, idx, k) : oz_b(P, B, k, idx - P.M); };
    constexpr unsigned long long MAG = 0x7fffffffffffffffull;
    unsigned long long mx = 0;
    for (int k = lane; k < P.K; k += 32) mx = max(mx, (unsigned long long)__double_as_longlong(val(k)) & MAG);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    // max |x| = 1.f 2^(ef - 1023) < 2^(ef - 1022); subnormal lines count as zero digits
    const int ef = (int)(mx >> 52);
    const int E = mx == 0 ? 0 : (ef == 0 ? -1021 : ef - 1022);
    if (lane == 0) ex[w] = E;
    const int Kp = oz_kp(P.K);
    uint32_t* out = (uint32_t*)(dig + eoff[np + 1 + lo] + (int64_t)idx * OZ_S * Kp);
    for (int k = 2 * lane; k < Kp; k += 64) {
        const double x0 = k < P.K ? val(k) : 0.0, x1 = k + 1 < P.K ? val(k + 1) : 0.0;
        oz_split2(x0, x1, E, out + k / 2, Kp / 2);
    }
}

__global__ void __launch_bounds__(OZ_NT, 2) gemm_oz_kernel(const GemmProb* __restrict__ probs, int np,
        const int64_t* __restrict__ eoff, const int* __restrict__ ex, const __nv_bfloat16* __restrict__ dig,
        double* Cb, const double* C0b)
{
    extern __shared__ __align__(16) unsigned char oz_smem[];
    __shared__ int eA[OZ_BM], eB[OZ_BN];
    const int64_t t = blockIdx.x;
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (probs[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    const GemmProb P = probs[lo];
    const int64_t lt = t - P.tile0;
    const int tm = (int)(lt % P.tiles_m), tn = (int)(lt / P.tiles_m);
    const int row0 = tm * OZ_BM, col0 = tn * OZ_BN;
    if (P.lower && col0 > row0 + OZ_BM - 1) return;          // wholly above the diagonal
    const int Kp = oz_kp(P.K);
    const __nv_bfloat16* digA = dig + eoff[np + 1 + lo];                  // line r: digA + r 8 Kp
    const __nv_bfloat16* digB = digA + (int64_t)P.M * OZ_S * Kp;
    const int* exA = ex + eoff[lo];
    const int* exB = exA + P.M;
    for (int e = threadIdx.x; e < OZ_BM; e += OZ_NT) eA[e] = row0 + e < P.M ? exA[row0 + e] : 0;
    for (int e = threadIdx.x; e < OZ_BN; e += OZ_NT) eB[e] = col0 + e < P.N ? exB[col0 + e] : 0;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp & 3) * 16, wn = (warp >> 2) * 16;   // the warp's 16 x 16 block of the tile
    const int g = lane >> 2, q = lane & 3;
    float S[OZ_S][2][4];                                      // level sums of the chunk, two n8 tiles
    long long WA[2][4], WB[2][4];
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
        for (int e = 0; e < 4; ++e) WA[n][e] = WB[n][e] = 0;
    auto zeroS = [&]() {
#pragma unroll
        for (int l = 0; l < OZ_S; ++l)
#pragma unroll
            for (int n = 0; n < 2; ++n)
#pragma unroll
                for (int e = 0; e < 4; ++e) S[l][n][e] = 0.0f;
    };
    auto flush = [&]() {                                      // the chunk's level sums into int64
#pragma unroll
        for (int n = 0; n < 2; ++n)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                long long a = 0, b = 0;
#pragma unroll
                for (int l = 0; l < 4; ++l) a = a * 128 + (long long)__float2int_rz(S[l][n][e]);
#pragma unroll
                for (int l = 4; l < 8; ++l) b = b * 128 + (long long)__float2int_rz(S[l][n][e]);
                WA[n][e] += a;
                WB[n][e] += b;
            }
    };
    // the digit tiles of stage st (16 k of 8 slices: 64 rows of A, 32 columns of B) go to buffer
    // st & 1 by cp.async, two 16-byte pieces per slice and line, zero fill outside the matrices;
    // stage st + 1 is in flight while stage st's products run
    auto issue = [&](int st, int buf) {
        const int k0 = st * OZ_BK;
        __nv_bfloat16* sb = reinterpret_cast<__nv_bfloat16*>(oz_smem) + buf * OZ_BUF;
        for (int e = threadIdx.x; e < OZ_S * (OZ_BM + OZ_BN) * 2; e += OZ_NT) {
            const int sl = e / ((OZ_BM + OZ_BN) * 2), rem = e - sl * (OZ_BM + OZ_BN) * 2;
            const int line = rem >> 1, c = rem & 1;
            const bool isA = line < OZ_BM;
            const int gl = isA ? row0 + line : col0 + line - OZ_BM;
            const bool ok = gl < (isA ? P.M : P.N);
            const __nv_bfloat16* src = (isA ? digA : digB) + (ok ? (int64_t)gl * OZ_S * Kp + sl * Kp + k0 + 8 * c : 0);
            __nv_bfloat16* dst = sb + (isA ? (sl * OZ_BM + line) : (OZ_S * OZ_BM + sl * OZ_BN + line - OZ_BM)) * OZ_LD + 8 * c;
            const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(ok ? 16 : 0));
        }
        asm volatile("cp.async.commit_group;");
    };
    zeroS();
    const int nst = (P.K + OZ_BK - 1) / OZ_BK;
    issue(0, 0);
    for (int st = 0; st < nst; ++st) {
        const int k0 = st * OZ_BK;
        if (st + 1 < nst) {
            issue(st + 1, (st + 1) & 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();                 // stage st landed in every thread's view
        auto As = reinterpret_cast<__nv_bfloat16 (*)[OZ_BM][OZ_LD]>(oz_smem + sizeof(__nv_bfloat16) * (st & 1) * OZ_BUF);
        auto Bs = reinterpret_cast<__nv_bfloat16 (*)[OZ_BN][OZ_LD]>(oz_smem + sizeof(__nv_bfloat16) *
                                                                    ((st & 1) * OZ_BUF + OZ_S * OZ_BM * OZ_LD));
#pragma unroll
        for (int ks = 0; ks < OZ_BK; ks += 16) {
            // A slices in the order 7, 0, 4, 1, 5, 2, 6, 3 (compile-time, so the level sums stay in
            // registers): with the B slices ascending inside, two products into the same level
            // sum are at least two pairs apart
            auto slice = [&](auto Ic) {
                constexpr int i = decltype(Ic)::value;
                uint32_t a[4];
                a[0] = *(const uint32_t*)&As[i][wm + g][ks + 2 * q];
                a[1] = *(const uint32_t*)&As[i][wm + g + 8][ks + 2 * q];
                a[2] = *(const uint32_t*)&As[i][wm + g][ks + 2 * q + 8];
                a[3] = *(const uint32_t*)&As[i][wm + g + 8][ks + 2 * q + 8];
#pragma unroll
                for (int j = 0; j + i < OZ_S; ++j) {
#pragma unroll
                    for (int n = 0; n < 2; ++n) {
                        const uint32_t b0 = *(const uint32_t*)&Bs[j][wn + 8 * n + g][ks + 2 * q];
                        const uint32_t b1 = *(const uint32_t*)&Bs[j][wn + 8 * n + g][ks + 2 * q + 8];
                        oz_mma(S[i + j][n], a, b0, b1);
                    }
                }
            };
            slice(std::integral_constant<int, 7>{});
            slice(std::integral_constant<int, 0>{});
            slice(std::integral_constant<int, 4>{});
            slice(std::integral_constant<int, 1>{});
            slice(std::integral_constant<int, 5>{});
            slice(std::integral_constant<int, 2>{});
            slice(std::integral_constant<int, 6>{});
            slice(std::integral_constant<int, 3>{});
        }
        __syncthreads();                 // buffer st & 1 is free for stage st + 2
        if ((k0 + OZ_BK) % OZ_CHUNK == 0 || k0 + OZ_BK >= P.K) {
            flush();
            zeroS();
        }
    }
    // C = alpha 2^(EA+EB-35) (W_A + 2^-28 W_B) + beta C0
    double* C = Cb + P.c_off;
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int li = wm + g + (e >= 2 ? 8 : 0), lj = wn + 8 * n + 2 * q + (e & 1);
            const int gi = row0 + li, gj = col0 + lj;
            if (gi >= P.M || gj >= P.N) continue;
            // the one FP64 operation per entry is the update's addition (alpha = +-1, beta = 0 or 1
            // in this library's products)
            double val = oz_round(WA[n][e], WB[n][e], eA[li] + eB[lj] - 63);
            if (P.alpha == -1.0) val = -val;
            else if (P.alpha != 1.0) val *= P.alpha;
            double out = val;
            if (P.beta != 0.0) {
                const double c0 = C0b[P.c0_off + (int64_t)gj * P.ldc0 + gi];
                out = P.beta == 1.0 ? c0 + val : fma(P.beta, c0, val);
            }
            C[(int64_t)gj * P.ldc + gi] = out;
        }
}

}  // namespace

OzPlan gemm_oz_plan(std::vector<GemmProb>& probs, std::vector<int64_t>& eoff)
{
    const size_t np = probs.size();
    OzPlan pl{0, 0, 0};
    eoff.assign(2 * (np + 1), 0);
    for (size_t p = 0; p < np; ++p) {
        GemmProb& g = probs[p];
        g.tiles_m = (g.M + OZ_BM - 1) / OZ_BM;
        g.tiles_n = (g.N + OZ_BN - 1) / OZ_BN;
        g.tile0 = pl.tiles;
        pl.tiles += (int64_t)g.tiles_m * g.tiles_n;
        eoff[p + 1] = eoff[p] + g.M + g.N;
        eoff[np + 2 + p] = eoff[np + 1 + p] + (int64_t)(g.M + g.N) * OZ_S * oz_kp(g.K);
    }
    pl.lines = eoff[np];
    pl.digits = eoff[2 * np + 1];
    return pl;
}

cudaError_t launch_gemm_oz(cudaStream_t st, const GemmProb* probs, int np, const OzPlan& pl, const int64_t* eoff,
                           int* ex, void* digits, const double* A, const double* B, double* C, const double* C0)
{
    if (np <= 0 || pl.tiles <= 0) return cudaSuccess;
    count_launches(2);
    __nv_bfloat16* dig = (__nv_bfloat16*)digits;
    oz_split_kernel<<<(unsigned)((pl.lines * 32 + 255) / 256), 256, 0, st>>>(probs, np, eoff, pl.lines, A, B, ex, dig);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    constexpr int shm = (int)(sizeof(__nv_bfloat16) * 2 * OZ_BUF);
    e = cudaFuncSetAttribute(gemm_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, shm);
    if (e != cudaSuccess) return e;
    gemm_oz_kernel<<<(unsigned)pl.tiles, OZ_NT, shm, st>>>(probs, np, eoff, ex, dig, C, C0);
    return cudaGetLastError();
}

}  // namespace rs
