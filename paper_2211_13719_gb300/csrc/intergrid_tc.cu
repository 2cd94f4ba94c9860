// Restriction and prolongation on the tensor cores (paper Sec. 5): FP16
// operands, FP32 accumulation in tensor memory, up to 32 null vectors and
// 64 RHS.  Used by the V-cycle of hierarchies built with a 16-bit coarse
// precision; the FP32 CUDA-core versions (mg.cu) build the Galerkin operator.
//
// Per aggregate and chirality chi the prolongator block P (R x N complex,
// R = sites x dof/2 rows rho) enters both products once, as [Re P | Im P]:
//
//   prolongation  psi_rho[r] = sum_k P[rho][k] c[k][r]
//     D = [Re P | Im P] (R x 2N) . [[Re c, Im c], [-Im c, Re c]] (2N x 2n)
//     Re psi = D[:, r], Im psi = D[:, n + r];   M = 128 rows per tile, K = 64.
//   restriction   c[k][r] = sum_rho conj(P[rho][k]) psi_rho[r]
//     D' = [Re psi | Im psi]^T (2n x R) . [Re P | Im P] (R x 2N)
//     Re c = D'[r][k] + D'[n+r][N+k], Im c = D'[n+r][k] - D'[r][N+k];
//     M = 128 RHS rows (2n padded), N = 64, K = R in chunks of 64.
//
// The P tiles are packed once at setup into the 128-byte-swizzled K-major
// image the MMA descriptors describe and arrive in shared memory by bulk
// copies on mbarriers; the field-side tiles are built by the CTA's threads
// from the FP32 fields, multiplied by one factor per RHS column (from a bound
// on the column's largest component: 1 for the unit-norm vectors of the
// V-cycle, the measured maximum otherwise; for prolongation the maximum over
// the aggregate's coarse block), and made visible to the tensor cores with
// fence.proxy.async.  One CTA per (aggregate, chirality); thread 0 issues the
// MMAs and commits them to mbarriers; every wait is bounded and on expiry the
// kernel records an error flag, stops issuing, waits (bounded) for its copies
// and MMAs, frees tensor memory and returns.
#include <algorithm>
#include <type_traits>

#include "mg.cuh"
#include "tc_common.cuh"

namespace mrhs {

namespace {

using namespace tc;

constexpr int IG_ROWS = 128;              // MMA M
constexpr int IG_K = 64;                  // one swizzle atom of 16-bit values
constexpr int IG_TILE = IG_ROWS * IG_K * 2;  // 16 KB
constexpr int IG_BTILE = 64 * IG_K * 2;      // 8 KB (restriction: 64 columns of P)
// scale of the lo parts of split-precision operands: the rounding error of an FP16 number is at
// most 2^-11 of it, so lo * 2^11 keeps the magnitude of hi and stays a normal FP16 number
constexpr float SPLIT_LO = 2048.f;

struct IgArgs {
    int L[4], Lc[4], B[4];
    int asize, dof, half, N, n, npad;
    int R;        // rows per chirality block: asize * half
    int tiles;    // prolongation: ceil(R / 128)
    int chunks;   // restriction: ceil(R / 64)
    int64_t ostride;  // restriction: coarse-site stride of the output
};

// fine site of local site s of aggregate xc (lexicographic inside the block)
__device__ __forceinline__ int64_t ig_site(const IgArgs &a, int64_t xc, int s) {
    int cc[4];
    site_to_coords(xc, a.Lc, cc);
    int f[4];
    f[0] = cc[0] * a.B[0] + s % a.B[0];
    int q = s / a.B[0];
    f[1] = cc[1] * a.B[1] + q % a.B[1];
    q /= a.B[1];
    f[2] = cc[2] * a.B[2] + q % a.B[2];
    f[3] = cc[3] * a.B[3] + q / a.B[2];
    return coords_to_site(f, a.L);
}

// value of [Re P | Im P] at row rho of chirality chi, column kp (zero padded)
__device__ __forceinline__ float pblock(const float2 *__restrict__ P, const IgArgs &a, int64_t xc, int chi, int rho,
                                        int kp) {
    if (rho >= a.R || kp >= 2 * a.N) return 0.f;
    const int s = rho / a.half, dl = rho - s * a.half;
    const int64_t x = ig_site(a, xc, s);
    const int k = kp < a.N ? kp : kp - a.N;
    const float2 v = P[(x * a.dof + chi * a.half + dl) * a.N + k];
    return kp < a.N ? v.x : v.y;
}

// prolongation A tiles: [Vc][2][tiles] x (128 rows rho, 64 columns kp)
__global__ void k_pack_prolong_tiles(const float2 *__restrict__ P, uint8_t *__restrict__ img, IgArgs a, int64_t Vc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per_tile = (int64_t)IG_ROWS * IG_K;
    if (i >= Vc * 2 * a.tiles * per_tile) return;
    const int64_t tile = i / per_tile;
    const int rem = (int)(i - tile * per_tile);
    const int row = rem / IG_K, kp = rem - row * IG_K;
    const int t = (int)(tile % a.tiles);
    const int chi = (int)((tile / a.tiles) % 2);
    const int64_t xc = tile / (2 * a.tiles);
    const float v = pblock(P, a, xc, chi, t * IG_ROWS + row, kp);
    *reinterpret_cast<uint16_t *>(img + tile * IG_TILE + sw128_offset(row, kp)) = to16<0>(v);
}

// restriction B tiles: [Vc][2][chunks] x (64 rows kp, 64 columns rho)
// LO: the FP16 rounding error of each value instead, times 2^11 (SPLIT_LO), so that it stays a
// normal FP16 number: the second term of a split-precision product
template <bool LO>
__global__ void k_pack_restrict_tiles(const float2 *__restrict__ P, uint8_t *__restrict__ img, IgArgs a, int64_t Vc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per_tile = 64LL * IG_K;
    if (i >= Vc * 2 * a.chunks * per_tile) return;
    const int64_t tile = i / per_tile;
    const int rem = (int)(i - tile * per_tile);
    const int kp = rem / IG_K, rl = rem - kp * IG_K;
    const int c = (int)(tile % a.chunks);
    const int chi = (int)((tile / a.chunks) % 2);
    const int64_t xc = tile / (2 * a.chunks);
    const float v = pblock(P, a, xc, chi, c * IG_K + rl, kp);
    const float x = LO ? (v - __half2float(__float2half_rn(v))) * SPLIT_LO : v;
    *reinterpret_cast<uint16_t *>(img + tile * IG_BTILE + sw128_offset(kp, rl)) = to16<0>(x);
}

__device__ __forceinline__ void atomic_max_pos(unsigned *addr, float v) { atomicMax(addr, __float_as_uint(v)); }

// two floats rounded to FP16, lo in the low half
__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// hi = fp16 of two floats, lo = fp16 of their rounding errors times SPLIT_LO (halves: a low, b high)
__device__ __forceinline__ void split_half2(float a, float b, uint32_t &hi, uint32_t &lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn((a - hf.x) * SPLIT_LO, (b - hf.y) * SPLIT_LO);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

// rowoff[rho] = fine row index (site * dof + component) of row rho of (aggregate xc, chirality chi)
__device__ __forceinline__ void fill_rows(int *rowoff, const IgArgs &a, int64_t xc, int chi) {
    for (int rho = threadIdx.x; rho < a.R; rho += blockDim.x) {
        const int s = rho / a.half, dl = rho - s * a.half;
        rowoff[rho] = (int)(ig_site(a, xc, s) * a.dof + chi * a.half + dl);
    }
}

constexpr int IG_MAX_ROWS = 4096;  // rows per (aggregate, chirality) handled by the tensor-core transfers

// Field-side values enter the MMAs as FP16 after multiplication by
// IG_UNIT / bound[r], bound[r] >= max |component| of RHS column r, so every
// operand stays below 2^14 in magnitude (no FP16 overflow) while values down
// to 2^-28 bound[r] stay normal; the epilogue multiplies by bound[r] / IG_UNIT.
constexpr float IG_UNIT = 16384.f;

// ---------------------------------------------------------- prolongation
constexpr int IG_STAGES = 3;  // P tiles in flight per CTA

// smem: [B tile npad x 64 | A ring IG_STAGES x 128 x 64 | row table R ints].
// The output columns of D interleave Re and Im (2r: Re psi[r], 2r + 1: Im
// psi[r]), so tensor-memory lane rho holds fine row rho in memory order and
// each thread stores its own row.  Two accumulators: the MMAs of tile t + 1
// run while tile t is drained.  THR = 256 (an autotuner variant): the two
// warps of each tensor-memory lane quarter share a row's columns, twice the
// warps draining the store-bound epilogue.
template <int VEC, int THR>
__global__ void __launch_bounds__(THR) k_prolong_tc(const float2 *__restrict__ coarse,
                                                            const uint8_t *__restrict__ PA, float2 *__restrict__ fine,
                                                            IgArgs a, int *__restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full[IG_STAGES];  // the stage's P tile landed
    __shared__ uint64_t done[2];          // MMAs into accumulator b complete
    __shared__ uint32_t tmem_sh;
    __shared__ unsigned scale_bits[64];
    __shared__ float inv_s[64], out_s[64];
    __shared__ int abort_sh;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t xc = blockIdx.x;
    const int chi = blockIdx.y;
    const int n = a.n, N = a.N, nc = 2 * N;
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *Bt = base;
    const uint32_t bt_bytes = ((uint32_t)a.npad * 128u + 1023u) & ~1023u;
    uint8_t *At = base + bt_bytes;
    int *rowoff = reinterpret_cast<int *>(At + IG_STAGES * IG_TILE);
    const uint32_t acc_cols = a.npad <= 32 ? 32u : (a.npad <= 64 ? 64u : 128u);
    const uint32_t cols = 2 * acc_cols;

    fill_rows(rowoff, a, xc, chi);
    if (tid < 64) scale_bits[tid] = 0u;
    if (tid == 0) {
        for (int i = 0; i < IG_STAGES; ++i) mbar_init(smem_u32(&full[i]), 1);
        mbar_init(smem_u32(&done[0]), 1);
        mbar_init(smem_u32(&done[1]), 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_sh), cols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_sh;
    const uint8_t *pa = PA + ((xc * 2 + chi) * (int64_t)a.tiles) * IG_TILE;
    // thread 0's record of what it has in flight, for a clean exit after an expired wait
    int copies = 0, copies_waited = 0, mmas = 0;
    if (tid == 0) {
        for (int t = 0; t < IG_STAGES && t < a.tiles; ++t) {
            mbar_expect_tx(smem_u32(&full[t]), IG_TILE);
            bulk_g2s(smem_u32(At + t * IG_TILE), pa + (int64_t)t * IG_TILE, IG_TILE, smem_u32(&full[t]));
            ++copies;
        }
    }
    // per-RHS scale of this aggregate's coarse block (chirality chi): values enter
    // the MMA as c * IG_UNIT / max|c|
    const float2 *cb = coarse + (xc * nc + chi * N) * n;
    for (int i = tid; i < N * n; i += blockDim.x) {
        const float2 v = cb[i];
        atomic_max_pos(&scale_bits[i % n], fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    __syncthreads();
    if (tid < n) {
        const float sc = __uint_as_float(scale_bits[tid]);
        inv_s[tid] = sc > 0.f ? IG_UNIT / sc : 0.f;
        out_s[tid] = sc / IG_UNIT;
    }
    __syncthreads();
    // B^T tile: row j (2r: Re of output column r, 2r + 1: Im), column kp
    for (int i = tid; i < a.npad * IG_K; i += blockDim.x) {
        const int j = i / IG_K, kp = i - j * IG_K;
        float v = 0.f;
        if (j < 2 * n && kp < nc) {
            const int r = j >> 1;
            const bool re = (j & 1) == 0;
            const int k = kp < N ? kp : kp - N;
            const float2 c = cb[k * n + r];
            // rows kp < N multiply Re P: [Re c | Im c]; rows kp >= N multiply Im P: [-Im c | Re c]
            const float val = kp < N ? (re ? c.x : c.y) : (re ? -c.y : c.x);
            v = val * inv_s[r];
        }
        *reinterpret_cast<uint16_t *>(Bt + sw128_offset(j, kp)) = to16<0>(v);
    }
    fence_async_smem();
    __syncthreads();

    const uint32_t idesc = idesc_16bit(IG_ROWS, a.npad, 0);
    // thread 0: MMAs of tile t into accumulator t & 1; false when its P tile never landed
    auto issue = [&](int t) -> bool {
        const int st = t % IG_STAGES;
        if (!mbar_wait(smem_u32(&full[st]), (t / IG_STAGES) & 1)) return false;
        ++copies_waited;
        fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(t & 1) * acc_cols;
#pragma unroll
        for (int kk = 0; kk < IG_K / 16; ++kk)
            mma_16bit(d, sdesc(smem_u32(At + st * IG_TILE) + kk * 32), sdesc(smem_u32(Bt) + kk * 32), idesc,
                      kk > 0 ? 1u : 0u);
        mma_commit(smem_u32(&done[t & 1]));
        ++mmas;
        return true;
    };
    if (tid == 0 && a.tiles > 0 && !issue(0)) abort_sh = 1;
    for (int t = 0; t < a.tiles; ++t) {
        // accumulator (t + 1) & 1 was drained in tile t - 1
        if (tid == 0 && !abort_sh && t + 1 < a.tiles && !issue(t + 1)) abort_sh = 1;
        if (!mbar_wait(smem_u32(&done[t & 1]), (t >> 1) & 1)) abort_sh = 1;
        __syncthreads();
        if (abort_sh) break;
        // stage t % IG_STAGES was read by tile t's MMAs, now complete
        if (tid == 0 && t + IG_STAGES < a.tiles) {
            const int st = t % IG_STAGES;
            mbar_expect_tx(smem_u32(&full[st]), IG_TILE);
            bulk_g2s(smem_u32(At + st * IG_TILE), pa + (int64_t)(t + IG_STAGES) * IG_TILE, IG_TILE,
                     smem_u32(&full[st]));
            ++copies;
        }
        fence_after_sync();
        const int q = warp & 3, grp = warp >> 2;  // lane quarter, column group
        const int rho = t * IG_ROWS + 32 * q + lane;
        float2 *dst = rho < a.R ? fine + (int64_t)rowoff[rho] * n : nullptr;
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(t & 1) * acc_cols;
        for (int c0 = 16 * grp; c0 < 2 * n; c0 += 16 * (THR / 128)) {
            float v[16];
            tmem_ld16(trow + (uint32_t)c0, v);
            if (!dst) continue;
            const int r0 = c0 >> 1;
            if (VEC == 2 && r0 + 8 <= n) {
                float4 *d4 = reinterpret_cast<float4 *>(dst + r0);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float s0 = out_s[r0 + 2 * i], s1 = out_s[r0 + 2 * i + 1];
                    __stcs(d4 + i, make_float4(v[4 * i] * s0, v[4 * i + 1] * s0, v[4 * i + 2] * s1, v[4 * i + 3] * s1));
                }
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int r = r0 + i;
                    if (r < n) __stcs(dst + r, make_float2(v[2 * i] * out_s[r], v[2 * i + 1] * out_s[r]));
                }
            }
        }
        fence_before_sync();
        __syncthreads();
    }
    if (abort_sh && tid == 0) {
        atomicExch(err, 1);
        // bounded: let copies and MMAs in flight land before the block exits
        for (int j = copies_waited; j < copies; ++j)
            mbar_wait(smem_u32(&full[j % IG_STAGES]), (j / IG_STAGES) & 1);
        if (mmas > 0) mbar_wait(smem_u32(&done[(mmas - 1) & 1]), ((mmas - 1) >> 1) & 1);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, cols);
}

// ----------------------------------------------------------- restriction

// smem: [A tiles 2 x NS x 128 x 64 (field) | B tiles 2 x NS x 64 x 64 (P) | row table R ints]
// (NS = 2 with SPLIT: hi and lo parts); the epilogue's D staging (128 x 65
// floats) reuses the A and B tiles.  Each thread loads all of its share of
// the next 64-row chunk into registers before it converts the current one.
//
// SPLIT (the Galerkin construction, where the result must keep FP32
// accuracy): every operand is the sum of two FP16 numbers, hi = fp16(x) and
// lo = fp16((x - hi) 2^11) 2^-11, 22 significant bits.  The product takes
// hi.hi into one FP32 accumulator and hi.lo + lo.hi into a second (the lo
// parts scaled by 2^11 stay normal FP16 numbers even where x is small); the
// epilogue adds acc0 + 2^-11 acc1.  The dropped lo.lo term is 2^-22 of the
// product.
template <int VEC, bool SPLIT>
__global__ void __launch_bounds__(128, 4) k_restrict_tc(const float2 *__restrict__ fine, const uint8_t *__restrict__ RB,
                                                     const uint8_t *__restrict__ RBlo,
                                                     float2 *__restrict__ coarse, const float *__restrict__ bound,
                                                     IgArgs a, int *__restrict__ err) {
    constexpr int NS = SPLIT ? 2 : 1;
    using LT = typename std::conditional<VEC == 2, float4, float2>::type;
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bars[4];  // [0, 1]: MMAs of buffer b complete; [2, 3]: B tile b landed
    __shared__ uint32_t tmem_sh;
    __shared__ float inv_s[64], out_s[64];
    __shared__ int abort_sh;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t xc = blockIdx.x;
    const int chi = blockIdx.y;
    const int n = a.n, N = a.N;
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *At = base;                  // buffer b, part h at At + (b * NS + h) * IG_TILE
    uint8_t *Bt = base + 2 * NS * IG_TILE;  // buffer b, part h at Bt + (b * NS + h) * IG_BTILE
    float *Ds = reinterpret_cast<float *>(base);
    constexpr int ld = 65;
    int *rowoff = reinterpret_cast<int *>(Bt + 2 * NS * IG_BTILE);
    constexpr uint32_t cols = SPLIT ? 128 : 64;  // SPLIT: acc0 at column 0, acc1 at column 64

    fill_rows(rowoff, a, xc, chi);
    if (tid < n) {
        const float b = bound[tid];
        inv_s[tid] = b > 0.f ? IG_UNIT / b : 0.f;
        out_s[tid] = b / IG_UNIT;
    }
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(smem_u32(&bars[i]), 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(smem_u32(&tmem_sh), cols);
    // rows j >= 2n of the A buffers stay zero
    for (int i = tid; i < 2 * NS * IG_TILE / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(At)[i] = make_uint4(0, 0, 0, 0);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_sh;

    // item v of a thread: 8-row group kc (one 16-byte chunk of the swizzled
    // A^T row) and column group p (VEC RHS); lanes with p >= n / VEC idle
    constexpr int PS = VEC == 2 ? 32 : 64;
    constexpr int ITEMS = 8 * PS / 128;
    const int np = n / VEC;
    LT buf[ITEMS][8];
    auto load_chunk = [&](int c) {
#pragma unroll
        for (int v = 0; v < ITEMS; ++v) {
            const int i = tid + 128 * v, kc = i / PS, p = i % PS;
            if (p >= np) continue;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int rho = c * IG_K + kc * 8 + j;
                if (rho < a.R) {
                    buf[v][j] = __ldcs(reinterpret_cast<const LT *>(fine + (int64_t)rowoff[rho] * n) + p);
                } else {
                    if constexpr (VEC == 2) buf[v][j] = make_float4(0.f, 0.f, 0.f, 0.f);
                    else buf[v][j] = make_float2(0.f, 0.f);
                }
            }
        }
    };
    // A^T tile: row r = Re of RHS column r, row n + r = Im, column = aggregate row of
    // the chunk; each item fills one 16-byte chunk (8 rows) of 2 VEC tile rows
    auto convert_chunk = [&](uint8_t *Ab) {
#pragma unroll
        for (int v = 0; v < ITEMS; ++v) {
            const int i = tid + 128 * v, kc = i / PS, p = i % PS;
            if (p >= np) continue;
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
                const int r = VEC * p + q;
                const float sc = inv_s[r];
                uint32_t re[4], im[4], rel[4], iml[4];
#pragma unroll
                for (int j = 0; j < 8; j += 2) {
                    float2 x0, x1;
                    if constexpr (VEC == 2) {
                        x0 = q == 0 ? make_float2(buf[v][j].x, buf[v][j].y) : make_float2(buf[v][j].z, buf[v][j].w);
                        x1 = q == 0 ? make_float2(buf[v][j + 1].x, buf[v][j + 1].y)
                                    : make_float2(buf[v][j + 1].z, buf[v][j + 1].w);
                    } else {
                        x0 = buf[v][j];
                        x1 = buf[v][j + 1];
                    }
                    if constexpr (SPLIT) {
                        split_half2(x0.x * sc, x1.x * sc, re[j / 2], rel[j / 2]);
                        split_half2(x0.y * sc, x1.y * sc, im[j / 2], iml[j / 2]);
                    } else {
                        re[j / 2] = pack_half2(x0.x * sc, x1.x * sc);
                        im[j / 2] = pack_half2(x0.y * sc, x1.y * sc);
                    }
                }
                *reinterpret_cast<uint4 *>(Ab + sw128_offset(r, 8 * kc)) = make_uint4(re[0], re[1], re[2], re[3]);
                *reinterpret_cast<uint4 *>(Ab + sw128_offset(n + r, 8 * kc)) = make_uint4(im[0], im[1], im[2], im[3]);
                if constexpr (SPLIT) {
                    uint8_t *Al = Ab + IG_TILE;
                    *reinterpret_cast<uint4 *>(Al + sw128_offset(r, 8 * kc)) = make_uint4(rel[0], rel[1], rel[2], rel[3]);
                    *reinterpret_cast<uint4 *>(Al + sw128_offset(n + r, 8 * kc)) =
                        make_uint4(iml[0], iml[1], iml[2], iml[3]);
                }
            }
        }
    };

    const uint32_t idesc = idesc_16bit(IG_ROWS, 64, 0);
    const uint8_t *rb = RB + ((xc * 2 + chi) * (int64_t)a.chunks) * IG_BTILE;
    const uint8_t *rbl = SPLIT ? RBlo + ((xc * 2 + chi) * (int64_t)a.chunks) * IG_BTILE : nullptr;
    // thread 0's record of what it has in flight, for a clean exit after an expired wait
    int copies = 0, copies_waited = 0, mmas = 0;
    load_chunk(0);
    for (int c = 0; c < a.chunks; ++c) {
        const int b = c & 1;
        if (c >= 1) {
            // buffers b were last read by the MMAs of chunk c - 2; an expired wait
            // of thread 0 in chunk c - 1 is seen here by every thread
            if (c >= 2 && !mbar_wait(smem_u32(&bars[b]), ((c - 2) >> 1) & 1)) abort_sh = 1;
            __syncthreads();
            if (abort_sh) break;
        }
        if (tid == 0) {
            mbar_expect_tx(smem_u32(&bars[2 + b]), NS * IG_BTILE);
            bulk_g2s(smem_u32(Bt + b * NS * IG_BTILE), rb + (int64_t)c * IG_BTILE, IG_BTILE, smem_u32(&bars[2 + b]));
            if constexpr (SPLIT)
                bulk_g2s(smem_u32(Bt + (b * NS + 1) * IG_BTILE), rbl + (int64_t)c * IG_BTILE, IG_BTILE,
                         smem_u32(&bars[2 + b]));
            ++copies;
        }
        convert_chunk(At + b * NS * IG_TILE);
        if (c + 1 < a.chunks) load_chunk(c + 1);
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            if (!mbar_wait(smem_u32(&bars[2 + b]), (c >> 1) & 1)) {
                abort_sh = 1;
            } else {
                ++copies_waited;
                fence_after_sync();
                const uint32_t a0 = smem_u32(At + b * NS * IG_TILE), b0 = smem_u32(Bt + b * NS * IG_BTILE);
#pragma unroll
                for (int kk = 0; kk < IG_K / 16; ++kk) {
                    mma_16bit(tmem, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), idesc, (c > 0 || kk > 0) ? 1u : 0u);
                    if constexpr (SPLIT) {
                        // the hi.lo and lo.hi terms, into the second accumulator
                        mma_16bit(tmem + 64, sdesc(a0 + kk * 32), sdesc(b0 + IG_BTILE + kk * 32), idesc,
                                  (c > 0 || kk > 0) ? 1u : 0u);
                        mma_16bit(tmem + 64, sdesc(a0 + IG_TILE + kk * 32), sdesc(b0 + kk * 32), idesc, 1u);
                    }
                }
                mma_commit(smem_u32(&bars[b]));
                ++mmas;
            }
        }
    }
    // the last commit covers every MMA issued before it
    if (!abort_sh && a.chunks > 0) {
        const int last = a.chunks - 1;
        if (!mbar_wait(smem_u32(&bars[last & 1]), (last >> 1) & 1)) abort_sh = 1;
    }
    __syncthreads();
    if (!abort_sh) {
        fence_after_sync();
        const int row = 32 * warp + (tid & 31);
        float v[4][16];
#pragma unroll
        for (int c0 = 0; c0 < 4; ++c0) tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(16 * c0), v[c0]);
        if constexpr (SPLIT) {
#pragma unroll
            for (int c0 = 0; c0 < 4; ++c0) {
                float u[16];
                tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(64 + 16 * c0), u);
#pragma unroll
                for (int i = 0; i < 16; ++i) v[c0][i] = fmaf(u[i], 1.f / SPLIT_LO, v[c0][i]);
            }
        }
        // the tile buffers are free: every MMA reading them has completed
#pragma unroll
        for (int c0 = 0; c0 < 4; ++c0)
#pragma unroll
            for (int i = 0; i < 16; ++i) Ds[row * ld + 16 * c0 + i] = v[c0][i];
        __syncthreads();
        for (int i = tid; i < N * n; i += blockDim.x) {
            const int k = i / n, r = i - k * n;
            const float sc = out_s[r];
            const float re = Ds[r * ld + k] + Ds[(n + r) * ld + N + k];
            const float im = Ds[(n + r) * ld + k] - Ds[r * ld + N + k];
            coarse[xc * a.ostride + (int64_t)(chi * N + k) * n + r] = make_float2(sc * re, sc * im);
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
        // bounded: let copies and MMAs in flight land before the block exits
        for (int j = copies_waited; j < copies; ++j) mbar_wait(smem_u32(&bars[2 + (j & 1)]), (j >> 1) & 1);
        if (mmas > 0) mbar_wait(smem_u32(&bars[(mmas - 1) & 1]), ((mmas - 1) >> 1) & 1);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, cols);
}

// per-column max |component| of a field [rows][n] (float bits compared as unsigned: valid for non-negative floats)
__global__ void k_field_absmax(const float2 *__restrict__ f, int64_t rows, int n, unsigned *__restrict__ col_max) {
    __shared__ unsigned sm[64];
    const int rpb = blockDim.x / n;
    const int col = threadIdx.x % n, rsub = threadIdx.x / n;
    if (threadIdx.x < 64) sm[threadIdx.x] = 0u;
    __syncthreads();
    if (rsub < rpb) {
        float m = 0.f;
        for (int64_t row = (int64_t)blockIdx.x * rpb + rsub; row < rows; row += (int64_t)gridDim.x * rpb) {
            const float2 v = __ldcs(f + row * n + col);
            m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
        atomic_max_pos(&sm[col], m);
    }
    __syncthreads();
    if (threadIdx.x < n) atomicMax(&col_max[threadIdx.x], sm[threadIdx.x]);
}

IgArgs ig_args(const Level &f, const Level &c, int n) {
    IgArgs a;
    for (int mu = 0; mu < 4; ++mu) {
        a.L[mu] = f.L[mu];
        a.Lc[mu] = c.L[mu];
        a.B[mu] = f.B[mu];
    }
    a.asize = (int)f.asize;
    a.dof = f.dof;
    a.half = f.dof / 2;
    a.N = f.N;
    a.n = n;
    a.npad = npad_of(n);
    a.R = a.asize * a.half;
    a.tiles = (a.R + IG_ROWS - 1) / IG_ROWS;
    a.chunks = (a.R + IG_K - 1) / IG_K;
    a.ostride = (int64_t)2 * f.N * n;
    return a;
}

constexpr int kProlongThreads[] = {128, 256};  // autotuner variants of the prolongation

size_t prolong_smem(int npad, int R) {
    const size_t bt = ((size_t)npad * 128 + 1023) & ~size_t(1023);
    return 1024 + bt + (size_t)IG_STAGES * IG_TILE + sizeof(int) * (size_t)R;
}
size_t restrict_smem(int R, bool split = false) {
    const size_t ns = split ? 2 : 1;
    return 1024 + 2 * ns * IG_TILE + 2 * ns * IG_BTILE + sizeof(int) * (size_t)R;
}

// 16-byte loads and stores of RHS pairs need an even n and a 16-byte aligned field
bool paired(const void *field, int n) { return n % 2 == 0 && (reinterpret_cast<uintptr_t>(field) & 15u) == 0; }

template <typename K> void allow_smem(K kernel, size_t bytes) {
    MRHS_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

}  // namespace

bool intergrid_tc_supported(const Level &f) { return f.N >= 1 && f.N <= 32 && f.asize * (f.dof / 2) <= IG_MAX_ROWS; }

void intergrid_tc_prepare(Level &f, const Level &c, cudaStream_t s, bool split) {
    if (!intergrid_tc_supported(f)) fail(MRHS_ERR_INVALID, "tensor-core intergrid needs at most 32 null vectors");
    const IgArgs a = ig_args(f, c, 1);
    if (split && !f.RBlo.ptr) {
        f.RBlo.alloc((size_t)c.V * 2 * a.chunks * IG_BTILE);
        const int64_t nr = c.V * 2 * a.chunks * 64LL * IG_K;
        k_pack_restrict_tiles<true><<<ceil_div(nr, 256), 256, 0, s>>>(f.P32.as<float2>(), f.RBlo.as<uint8_t>(), a,
                                                                       c.V);
        MRHS_LAUNCHED("k_pack_restrict_tiles");
    }
    if (f.PA.ptr) return;  // the tiles of this prolongator are packed already
    f.PA.alloc((size_t)c.V * 2 * a.tiles * IG_TILE);
    f.RB.alloc((size_t)c.V * 2 * a.chunks * IG_BTILE);
    f.IgErr.alloc(sizeof(int));
    f.IgBound.alloc(sizeof(float) * 128);
    zero_on_sms(f.IgErr.ptr, sizeof(int), s);
    static const float ones[64] = {1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f,
                                   1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f,
                                   1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f,
                                   1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f, 1.f};
    MRHS_CUDA(cudaMemcpyAsync(f.IgBound.ptr, ones, sizeof(ones), cudaMemcpyHostToDevice, s));
    const int64_t np = c.V * 2 * a.tiles * (int64_t)IG_ROWS * IG_K;
    k_pack_prolong_tiles<<<ceil_div(np, 256), 256, 0, s>>>(f.P32.as<float2>(), f.PA.as<uint8_t>(), a, c.V);
    MRHS_LAUNCHED("k_pack_prolong_tiles");
    const int64_t nr = c.V * 2 * a.chunks * 64LL * IG_K;
    k_pack_restrict_tiles<false><<<ceil_div(nr, 256), 256, 0, s>>>(f.P32.as<float2>(), f.RB.as<uint8_t>(), a, c.V);
    MRHS_LAUNCHED("k_pack_restrict_tiles");
    MRHS_CUDA(cudaStreamSynchronize(s));  // the host array of ones is copied before it can go out of scope
}

void restrict_fields_tc(const Level &f, const Level &c, const float2 *fine, float2 *coarse, int n, int64_t ostride,
                        bool unit_norm, cudaStream_t s, bool split) {
    if (!f.RB.ptr || (split && !f.RBlo.ptr)) fail(MRHS_ERR_INVALID, "tensor-core restriction not prepared");
    if (n < 1 || n > 64) fail(MRHS_ERR_INVALID, "tensor-core restriction supports 1..64 RHS");
    IgArgs a = ig_args(f, c, n);
    a.ostride = ostride;
    const float *bound = f.IgBound.as<float>();
    if (!unit_norm) {
        // bound[r] = max |component| of column r
        unsigned *cm = reinterpret_cast<unsigned *>(f.IgBound.as<float>() + 64);
        zero_on_sms(cm, sizeof(unsigned) * 64, s);
        const int64_t rows = f.rows();
        const int rpb = 256 / n;
        const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(sm_count(0) * 4, ceil_div(rows, 16LL * rpb)));
        k_field_absmax<<<blocks, 256, 0, s>>>(fine, rows, n, cm);
        MRHS_LAUNCHED("k_field_absmax");
        bound = f.IgBound.as<float>() + 64;
    }
    static bool attr = false;
    if (!attr) {
        allow_smem(k_restrict_tc<1, false>, restrict_smem(IG_MAX_ROWS));
        allow_smem(k_restrict_tc<2, false>, restrict_smem(IG_MAX_ROWS));
        allow_smem(k_restrict_tc<1, true>, restrict_smem(IG_MAX_ROWS, true));
        allow_smem(k_restrict_tc<2, true>, restrict_smem(IG_MAX_ROWS, true));
        attr = true;
    }
    const dim3 grid((unsigned)c.V, 2);
    const uint8_t *rb = f.RB.as<uint8_t>(), *rbl = f.RBlo.as<uint8_t>();
    const size_t smem = restrict_smem(a.R, split);
    MRHS_TIMED("k_restrict_tc", s);
    if (paired(fine, n)) {
        if (split) k_restrict_tc<2, true><<<grid, 128, smem, s>>>(fine, rb, rbl, coarse, bound, a, f.IgErr.as<int>());
        else k_restrict_tc<2, false><<<grid, 128, smem, s>>>(fine, rb, rbl, coarse, bound, a, f.IgErr.as<int>());
    } else {
        if (split) k_restrict_tc<1, true><<<grid, 128, smem, s>>>(fine, rb, rbl, coarse, bound, a, f.IgErr.as<int>());
        else k_restrict_tc<1, false><<<grid, 128, smem, s>>>(fine, rb, rbl, coarse, bound, a, f.IgErr.as<int>());
    }
    MRHS_LAUNCHED("k_restrict_tc");
}

void prolong_fields_tc(const Level &f, const Level &c, const float2 *coarse, float2 *fine, int n, cudaStream_t s) {
    if (!f.PA.ptr) fail(MRHS_ERR_INVALID, "tensor-core prolongation not prepared");
    if (n < 1 || n > 64) fail(MRHS_ERR_INVALID, "tensor-core prolongation supports 1..64 RHS");
    const IgArgs a = ig_args(f, c, n);
    static bool attr = false;
    if (!attr) {
        allow_smem(k_prolong_tc<1, 128>, prolong_smem(128, IG_MAX_ROWS));
        allow_smem(k_prolong_tc<2, 128>, prolong_smem(128, IG_MAX_ROWS));
        allow_smem(k_prolong_tc<1, 256>, prolong_smem(128, IG_MAX_ROWS));
        allow_smem(k_prolong_tc<2, 256>, prolong_smem(128, IG_MAX_ROWS));
        attr = true;
    }
    const dim3 grid((unsigned)c.V, 2);
    const size_t smem = prolong_smem(a.npad, a.R);
    const bool pr = paired(fine, n);
    auto launch = [&](int v) {
        const uint8_t *pa = f.PA.as<uint8_t>();
        int *err = f.IgErr.as<int>();
        if (kProlongThreads[v] == 256) {
            if (pr) k_prolong_tc<2, 256><<<grid, 256, smem, s>>>(coarse, pa, fine, a, err);
            else k_prolong_tc<1, 256><<<grid, 256, smem, s>>>(coarse, pa, fine, a, err);
        } else {
            if (pr) k_prolong_tc<2, 128><<<grid, 128, smem, s>>>(coarse, pa, fine, a, err);
            else k_prolong_tc<1, 128><<<grid, 128, smem, s>>>(coarse, pa, fine, a, err);
        }
        MRHS_CUDA(cudaGetLastError());
    };
    // the output overwrites `fine` from `coarse` alone: repeated launches are harmless
    const int v = tune_pick("k_prolong_tc", c.L, n, 2, launch, s);
    MRHS_TIMED("k_prolong_tc", s);
    launch(v);
    MRHS_LAUNCHED("k_prolong_tc");
}

int intergrid_tc_error(const Level &f, cudaStream_t s) {
    if (!f.IgErr.ptr) return 0;
    int *e = pinned_flag_slot();
    read_back(e, f.IgErr.ptr, sizeof(int), s);
    MRHS_CUDA(cudaStreamSynchronize(s));
    return *e;
}

}  // namespace mrhs
