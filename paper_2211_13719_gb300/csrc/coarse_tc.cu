// Coarse 9-point stencil on the 5th-generation tensor cores (paper Sec. 6):
// FP16 or BF16 operands, FP32 accumulation in tensor memory, nc = 64 coarse dof.
//
// Scaling: each site's 9 link blocks are stored divided by their largest
// real or imaginary component (one FP32 scale per site) and the input field
// is packed divided by its largest component per RHS column (one scale per
// column, found by a max-reduction before packing); both scales factor out
// of the site's sum and are applied to the FP32 result.  FP16 (11-bit
// significand) therefore neither overflows nor loses small magnitudes.
//
// Per coarse site x the stencil is one complex GEMM over the RHS block,
//   out[K][r] = sum_{d=0..8} sum_L A_d(x)[K][L] phi(x + delta_d)[L][r],
// computed as one real GEMM without duplicating the links: with
//   A'_d = [Re A_d ; Im A_d]        (128 x 64, rows K and 64 + K)
//   B_d  = [Re phi_d | Im phi_d]    (64 x 2n)
// D = sum_d A'_d B_d (128 x 2n) holds Re A Re phi, Re A Im phi, Im A Re phi
// and Im A Im phi, so
//   Re out[K][r] = D[K][r] - D[64+K][n+r],   Im out[K][r] = D[64+K][r] + D[K][n+r].
// M = 128, N = 2n rounded up to a multiple of 16, K = 9 * 64 (36 MMAs of K = 16).
//
// Operands sit in shared memory in the 128-byte-swizzled K-major layout the
// MMA descriptors describe (8-row atoms of 1024 bytes, 16-byte chunk c of
// row r stored at chunk c ^ (r % 8)).  Links are converted once into that
// image in global memory, so each (site, direction) tile is one contiguous
// 16 KB bulk copy; the neighbour fields are packed into the same image form
// by a small kernel before each apply.  One CTA per coarse site: a single
// thread issues the bulk copies through a 3-stage mbarrier ring and the
// MMAs; all four warps then read the accumulator out of tensor memory,
// recombine real and imaginary parts and store the FP32 result.
//
// Every wait on an mbarrier is bounded; on expiry the kernel records an
// error flag, drains its outstanding copies (bounded), frees its tensor
// memory and returns.  The host reads the flag after every standalone apply
// and during a solve, and turns it into MRHS_ERR_TIMEOUT.  For tests,
// mrhs_debug_expire_waits makes the first operand wait of the next launches
// give up at once (zero try_wait rounds); the drain then still waits for
// every copy already issued, so nothing is left in flight.
#include <algorithm>
#include <atomic>

#include "mg.cuh"
#include "tc_common.cuh"

namespace mrhs {
mrhs_status api_record(mrhs_status code, const std::string &msg);

namespace {

// launches (outside stream capture) whose first operand wait is to expire at once
std::atomic<int> g_expire_waits{0};

using namespace tc;

constexpr int NC = 64;                 // coarse dof handled by this kernel
constexpr int MROWS = 128;             // 2 * NC real rows
constexpr int A_TILE = MROWS * NC * 2; // bytes of one BF16 link tile (16 KB)
// depth of the bulk-copy ring (autotuner variants: 3, 2, 4 stages; fewer
// stages leave room for more CTAs per SM)
constexpr int kStageVariants[] = {3, 2, 4};

struct TcArgs {
    int L[4];
    int64_t V;
    int n, npad;
    uint32_t idesc;
    uint32_t tmem_cols;
    uint32_t first_limit;  // try_wait rounds of the first operand wait (SPIN_LIMIT; 0 when a test expires it)
    // stencil terms and site set: directions d_first..d_last; link tile of (site, d) at
    // site * links_per_site + d - d_first; parity < 0: every site, fields full-lattice;
    // parity 0 / 1: the output sites are those of that parity and the output field and
    // the packed input are half-lattice fields (a site s at index s / 2)
    int d_first, d_last;
    int links_per_site;
    int parity;
};

// site of half-lattice index cb and parity p (even x extent: the sites 2 cb and
// 2 cb + 1 form an x pair of opposite parities)
__device__ __forceinline__ int64_t cb_site(int64_t cb, int p, const int L[4]) {
    int c[4];
    site_to_coords(2 * cb, L, c);
    return ((c[0] + c[1] + c[2] + c[3]) & 1) == p ? 2 * cb : 2 * cb + 1;
}

template <int STAGES>
__global__ void __launch_bounds__(128) k_coarse_tc(const uint8_t *__restrict__ Abf, const uint8_t *__restrict__ Phi,
                                                   float2 *__restrict__ out, const float2 *__restrict__ y, TcArgs a,
                                                   const float *__restrict__ link_scale,
                                                   const float *__restrict__ col_scale, int *__restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t bars[2 * STAGES + 1];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_sh;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t cta = blockIdx.x;
    const int64_t site = a.parity < 0 ? cta : cb_site(cta, a.parity, a.L);
    const int ndir = a.d_last - a.d_first + 1;
    const uint32_t b_tile = (uint32_t)a.npad * 128u;
    const uint32_t stage_bytes = A_TILE + ((b_tile + 1023u) & ~1023u);
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(base);
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[STAGES]), done = smem_u32(&bars[2 * STAGES]);

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(a.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_sh;

    if (tid == 0) {
        // producer + MMA issuer: loads run STAGES - 1 directions ahead of the MMAs
        bool ok = true;
        int issued = 0;
        for (int step = 0; step < ndir + STAGES - 1 && ok; ++step) {
            if (step < ndir) {
                const int q = step, s = q % STAGES;
                if (q >= STAGES) ok = mbar_wait(empty0 + 8 * s, ((q / STAGES) - 1) & 1);
                if (!ok) break;
                const int d = a.d_first + q;
                const int64_t nb = stencil_nb_site(site, a.L, d);
                const int64_t pin = a.parity < 0 ? nb : nb >> 1;
                const uint32_t sa = sbase + s * stage_bytes;
                mbar_expect_tx(full0 + 8 * s, A_TILE + b_tile);
                bulk_g2s(sa, Abf + ((size_t)site * a.links_per_site + q) * A_TILE, A_TILE, full0 + 8 * s);
                bulk_g2s(sa + A_TILE, Phi + (size_t)pin * b_tile, b_tile, full0 + 8 * s);
                ++issued;
            }
            const int e = step - (STAGES - 1);
            if (e >= 0 && e < ndir) {
                const int s = e % STAGES;
                ok = mbar_wait_n(full0 + 8 * s, (e / STAGES) & 1, e == 0 ? a.first_limit : SPIN_LIMIT);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = sbase + s * stage_bytes, sb = sa + A_TILE;
#pragma unroll
                for (int kk = 0; kk < NC / 16; ++kk)
                    mma_16bit(tmem, sdesc(sa + kk * 32), sdesc(sb + kk * 32), a.idesc, (e > 0 || kk > 0) ? 1u : 0u);
                mma_commit(empty0 + 8 * s);
            }
        }
        if (ok) {
            mma_commit(done);
        } else {
            atomicExch(err, 1);
            abort_sh = 1;
            // drain: every issued stage's copies must land, and every issued MMA
            // finish, before the CTA frees its tensor memory and exits
            for (int d = 0; d < issued; ++d) mbar_wait(full0 + 8 * (d % STAGES), (d / STAGES) & 1);
            mma_commit(done);
            mbar_wait(done, 0);
        }
    }
    __syncthreads();
    bool ok = abort_sh == 0;
    if (ok) ok = mbar_wait(done, 0);
    if (!ok && tid == 0) atomicExch(err, 1);
    __syncthreads();
    if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // TMEM rows 32*warp .. 32*warp+31 -> shared staging D[row][col] (stage buffers are free now)
        float *Ds = reinterpret_cast<float *>(base);
        const int ld = a.npad + 1;
        const int row = 32 * warp + (tid & 31);
        for (int c0 = 0; c0 < a.npad; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) Ds[row * ld + c0 + i] = v[i];
        }
        __syncthreads();
        const int n = a.n;
        const float ls = link_scale[site];
        for (int idx = tid; idx < NC * n; idx += blockDim.x) {
            const int K = idx / n, r = idx - K * n;
            const float sc = ls * col_scale[r];
            float re = sc * (Ds[K * ld + r] - Ds[(NC + K) * ld + n + r]);
            float im = sc * (Ds[(NC + K) * ld + r] + Ds[K * ld + n + r]);
            const int64_t o = cta * (int64_t)(NC * n) + idx;
            if (y) {
                const float2 yy = y[o];
                re = yy.x - re;
                im = yy.y - im;
            }
            out[o] = make_float2(re, im);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols));
}

// per-RHS scale of the input: col_scale[r] = max over sites and components of
// max(|Re|, |Im|) (float bits compared as unsigned: valid for non-negative
// floats).  One column per thread, rows strided over the block and grid.
__global__ void k_col_absmax(const float2 *__restrict__ phi, int64_t rows, int n, unsigned *__restrict__ col_max) {
    __shared__ unsigned sm[64];
    const int rpb = blockDim.x / n;
    const int col = threadIdx.x % n, rsub = threadIdx.x / n;
    if (threadIdx.x < 64) sm[threadIdx.x] = 0u;
    __syncthreads();
    if (rsub < rpb) {
        float m = 0.f;
        for (int64_t row = (int64_t)blockIdx.x * rpb + rsub; row < rows; row += (int64_t)gridDim.x * rpb) {
            const float2 v = phi[row * n + col];
            m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
        atomicMax(&sm[col], __float_as_uint(m));
    }
    __syncthreads();
    if (threadIdx.x < n) atomicMax(&col_max[threadIdx.x], sm[threadIdx.x]);
}

// coarse field [V][64][n] FP32 -> per-site swizzled 16-bit image of [Re phi | Im phi]^T / col_scale.
// One CTA per site: coalesced reads of the site's 64 x n values, the tile is
// built in shared memory and written out with 16-byte stores.
template <int FMT>
__global__ void k_pack_phi(const float2 *__restrict__ phi, uint8_t *__restrict__ img, int n, int npad,
                           const float *__restrict__ col_scale) {
    extern __shared__ uint4 tile4[];
    __shared__ float inv[64];
    uint8_t *tile = reinterpret_cast<uint8_t *>(tile4);
    const int64_t site = blockIdx.x;
    const int tid = threadIdx.x;
    const int words = npad * 128 / 16;
    for (int i = tid; i < words; i += blockDim.x) tile4[i] = make_uint4(0, 0, 0, 0);
    if (tid < n) {
        const float c = col_scale[tid];
        inv[tid] = c > 0.f ? 1.f / c : 0.f;
    }
    __syncthreads();
    const float2 *src = phi + site * NC * n;
    for (int e = tid; e < NC * n; e += blockDim.x) {
        const int k = e / n, r = e - k * n;
        const float2 p = src[e];
        const float c = inv[r];
        *reinterpret_cast<uint16_t *>(tile + sw128_offset(r, k)) = to16<FMT>(p.x * c);
        *reinterpret_cast<uint16_t *>(tile + sw128_offset(n + r, k)) = to16<FMT>(p.y * c);
    }
    __syncthreads();
    uint4 *dst = reinterpret_cast<uint4 *>(img + site * (int64_t)npad * 128);
    for (int i = tid; i < words; i += blockDim.x) dst[i] = tile4[i];
}

// per-site scale of the links: max over the site's `tps` blocks of max(|Re|, |Im|)
__global__ void k_link_scale(const float2 *__restrict__ A, float *__restrict__ scale, int tps) {
    __shared__ float red[32];
    const int64_t site = blockIdx.x;
    const float2 *a = A + site * tps * NC * NC;
    float m = 0.f;
    for (int i = threadIdx.x; i < tps * NC * NC; i += blockDim.x) {
        const float2 v = a[i];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
        scale[site] = t > 0.f ? t : 1.f;
    }
}

// links [V][tps][64][64] complex FP32 -> [V][tps] swizzled 16-bit tiles of [Re A ; Im A] / scale (128 x 64)
template <int FMT>
__global__ void k_pack_links(const float2 *__restrict__ A, uint8_t *__restrict__ img, int64_t V,
                             const float *__restrict__ scale, int tps) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V * tps * MROWS * NC) return;
    const int64_t tile = i / (MROWS * NC);
    const int rem = (int)(i - tile * MROWS * NC);
    const int m = rem / NC, k = rem - m * NC;
    const float2 v = A[(tile * NC + (m % NC)) * NC + k];
    const float s = scale[tile / tps];
    *reinterpret_cast<uint16_t *>(img + tile * (int64_t)A_TILE + sw128_offset(m, k)) = to16<FMT>((m < NC ? v.x : v.y) / s);
}

size_t tc_smem_bytes(int npad, int stages) {
    const size_t b_tile = (size_t)npad * 128;
    const size_t stage = A_TILE + ((b_tile + 1023) & ~size_t(1023));
    const size_t epi = (size_t)MROWS * (npad + 1) * sizeof(float);
    return std::max(stage * stages, epi) + 1024;
}

}  // namespace

bool coarse_bf16_supported(const Level &c) { return c.dof == NC; }

uint32_t tc_first_wait_limit(cudaStream_t s) {
    // a launch recorded into a graph would keep the expired limit for every replay: only eager launches
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    MRHS_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return SPIN_LIMIT;
    int left = g_expire_waits.load();
    while (left > 0 && !g_expire_waits.compare_exchange_weak(left, left - 1)) {
    }
    return left > 0 ? 0u : SPIN_LIMIT;
}

void coarse_links_to_16bit(Level &c, mrhs_precision fmt, cudaStream_t s) {
    if (!coarse_bf16_supported(c)) fail(MRHS_ERR_INVALID, "16-bit tensor-core stencil needs 64 coarse dof");
    if (fmt != MRHS_FP16 && fmt != MRHS_BF16) fail(MRHS_ERR_INVALID, "16-bit format must be FP16 or BF16");
    c.tc_fmt = fmt;
    c.Abf.alloc((size_t)c.V * 9 * A_TILE);
    c.PhiBf.alloc((size_t)c.V * npad_of(64) * 128);
    c.TcErr.alloc(sizeof(int));
    c.LinkScale.alloc(sizeof(float) * (size_t)c.V);
    c.ColScale.alloc(sizeof(float) * 64);
    zero_on_sms(c.TcErr.ptr, sizeof(int), s);
    k_link_scale<<<(unsigned)c.V, 256, 0, s>>>(c.A32.as<float2>(), c.LinkScale.as<float>(), 9);
    MRHS_LAUNCHED("k_link_scale");
    const int64_t count = c.V * 9 * MROWS * NC;
    if (fmt == MRHS_FP16)
        k_pack_links<0><<<ceil_div(count, 256), 256, 0, s>>>(c.A32.as<float2>(), c.Abf.as<uint8_t>(), c.V,
                                                             c.LinkScale.as<float>(), 9);
    else
        k_pack_links<1><<<ceil_div(count, 256), 256, 0, s>>>(c.A32.as<float2>(), c.Abf.as<uint8_t>(), c.V,
                                                             c.LinkScale.as<float>(), 9);
    MRHS_LAUNCHED("k_pack_links");
}

// The tensor-core stencil in general form: out (n RHS, nc = 64) at the output
// sites of `parity` (every site for parity < 0) = sum over directions
// d_first..d_last of the link tiles `links` (links_per_site per site, scaled
// per site by link_scale) times the input at the site's neighbours (or y minus
// that).  `in` holds in_sites sites: the whole lattice for parity < 0, else the
// half field whose sites are the neighbours' parity.
void coarse_tc_general(const Level &c, const uint8_t *links, const float *link_scale, int links_per_site,
                       int d_first, int d_last, int parity, const float2 *in, int64_t in_sites, float2 *out,
                       const float2 *y, int n, cudaStream_t s) {
    if (!c.Abf.ptr) fail(MRHS_ERR_INVALID, "16-bit links not prepared");
    if (n < 1 || n > 64) fail(MRHS_ERR_INVALID, "tensor-core coarse stencil supports 1..64 RHS");
    const int npad = npad_of(n);
    zero_on_sms(c.ColScale.ptr, sizeof(float) * 64, s);
    const int64_t rows = in_sites * NC;
    const int rpb = 256 / n;
    const int ablocks = (int)std::max<int64_t>(1, std::min<int64_t>(sm_count(0) * 4, ceil_div(rows, 8LL * rpb)));
    k_col_absmax<<<ablocks, 256, 0, s>>>(in, rows, n, c.ColScale.as<unsigned>());
    MRHS_LAUNCHED("k_col_absmax");
    const size_t tile_bytes = (size_t)npad * 128;
    if (c.tc_fmt == MRHS_FP16)
        k_pack_phi<0><<<(unsigned)in_sites, 256, tile_bytes, s>>>(in, c.PhiBf.as<uint8_t>(), n, npad,
                                                                  c.ColScale.as<float>());
    else
        k_pack_phi<1><<<(unsigned)in_sites, 256, tile_bytes, s>>>(in, c.PhiBf.as<uint8_t>(), n, npad,
                                                                  c.ColScale.as<float>());
    MRHS_LAUNCHED("k_pack_phi");
    TcArgs a;
    for (int mu = 0; mu < 4; ++mu) a.L[mu] = c.L[mu];
    a.V = c.V;
    a.n = n;
    a.npad = npad;
    a.idesc = idesc_16bit(MROWS, npad, c.tc_fmt == MRHS_FP16 ? 0u : 1u);
    a.tmem_cols = npad <= 32 ? 32 : (npad <= 64 ? 64 : 128);
    a.first_limit = tc_first_wait_limit(s);
    a.d_first = d_first;
    a.d_last = d_last;
    a.links_per_site = links_per_site;
    a.parity = parity;
    static bool attr = false;
    if (!attr) {
        MRHS_CUDA(cudaFuncSetAttribute(k_coarse_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes(128, 2)));
        MRHS_CUDA(cudaFuncSetAttribute(k_coarse_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes(128, 3)));
        MRHS_CUDA(cudaFuncSetAttribute(k_coarse_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes(128, 4)));
        attr = true;
    }
    const int64_t out_sites = parity < 0 ? c.V : c.V / 2;
    auto launch = [&](int v) {
        const int stages = kStageVariants[v];
        const size_t smem = tc_smem_bytes(npad, stages);
        auto go = [&](auto kern) {
            kern<<<(unsigned)out_sites, 128, smem, s>>>(links, c.PhiBf.as<uint8_t>(), out, y, a, link_scale,
                                                        c.ColScale.as<float>(), c.TcErr.as<int>());
        };
        if (stages == 2) go(k_coarse_tc<2>);
        else if (stages == 4) go(k_coarse_tc<4>);
        else go(k_coarse_tc<3>);
        MRHS_CUDA(cudaGetLastError());
    };
    // an output that aliases an input would not survive repeated launches; an expiring
    // wait must happen in the launch that is not repeated: no tuning then.  The tuner
    // key holds the level's extents; the even-odd forms tune under their own names.
    const bool alias = (const void *)out == (const void *)in || (y && (const void *)out == (const void *)y);
    static const char *names[] = {"k_coarse_tc", "k_coarse_tc_eo_hop", "k_coarse_tc_eo_self"};
    const char *name = parity < 0 ? names[0] : (d_first > 0 ? names[1] : names[2]);
    const int v = (alias || a.first_limit == 0) ? 0 : tune_pick(name, c.L, n, 3, launch, s);
    MRHS_TIMED("k_coarse_tc", s);
    launch(v);
    MRHS_LAUNCHED("k_coarse_tc");
}

void coarse_apply_bf16(const Level &c, const float2 *in, float2 *out, const float2 *y, int n, cudaStream_t s) {
    if (!c.Abf.ptr) fail(MRHS_ERR_INVALID, "16-bit links not prepared");
    coarse_tc_general(c, c.Abf.as<uint8_t>(), c.LinkScale.as<float>(), 9, 0, 8, -1, in, c.V, out, y, n, s);
}

// ------------------------------------------- coarse even-odd (Sec. 6, M_eooe)
namespace {

// Inverse of the self block A_0(x) of every coarse site: Gauss-Jordan with
// partial pivoting in FP64 on [A_0 | 1] in shared memory (64 x 128 complex), one
// CTA per site; a pivot below 1e-300 (singular block) sets *singular.
__global__ void __launch_bounds__(256) k_self_inverse(const float2 *__restrict__ A, float2 *__restrict__ inv,
                                                      int *__restrict__ singular) {
    extern __shared__ double2 M[];  // [64][128]
    __shared__ double2 fac[NC];
    __shared__ int piv_sh;
    __shared__ double best_sh;
    const int64_t site = blockIdx.x;
    const float2 *a0 = A + site * 9 * NC * NC;  // direction 0
    for (int e = threadIdx.x; e < NC * 2 * NC; e += blockDim.x) {
        const int r = e / (2 * NC), j = e - r * 2 * NC;
        if (j < NC) {
            const float2 v = a0[r * NC + j];
            M[e] = make_double2(v.x, v.y);
        } else {
            M[e] = make_double2(j - NC == r ? 1.0 : 0.0, 0.0);
        }
    }
    __syncthreads();
    for (int col = 0; col < NC; ++col) {
        if (threadIdx.x == 0) {
            int piv = col;
            double best = -1.0;
            for (int r = col; r < NC; ++r) {
                const double2 v = M[r * 2 * NC + col];
                const double m = v.x * v.x + v.y * v.y;
                if (m > best) {
                    best = m;
                    piv = r;
                }
            }
            piv_sh = piv;
            best_sh = best;
            if (!(best > 1e-300)) atomicExch(singular, 1);
        }
        __syncthreads();
        if (!(best_sh > 1e-300)) return;
        const int piv = piv_sh;
        if (piv != col)
            for (int j = threadIdx.x; j < 2 * NC; j += blockDim.x) {
                const double2 t = M[col * 2 * NC + j];
                M[col * 2 * NC + j] = M[piv * 2 * NC + j];
                M[piv * 2 * NC + j] = t;
            }
        __syncthreads();
        const double2 p = M[col * 2 * NC + col];
        const double pm = p.x * p.x + p.y * p.y;
        const double2 pinv = make_double2(p.x / pm, -p.y / pm);
        __syncthreads();
        for (int j = threadIdx.x; j < 2 * NC; j += blockDim.x) {
            const double2 v = M[col * 2 * NC + j];
            M[col * 2 * NC + j] = make_double2(v.x * pinv.x - v.y * pinv.y, v.x * pinv.y + v.y * pinv.x);
        }
        __syncthreads();
        if (threadIdx.x < NC) fac[threadIdx.x] = M[threadIdx.x * 2 * NC + col];
        __syncthreads();
        for (int e = threadIdx.x; e < NC * 2 * NC; e += blockDim.x) {
            const int r = e / (2 * NC), j = e - r * 2 * NC;
            if (r == col) continue;
            const double2 f = fac[r], u = M[col * 2 * NC + j];
            double2 v = M[e];
            v.x -= f.x * u.x - f.y * u.y;
            v.y -= f.x * u.y + f.y * u.x;
            M[e] = v;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < NC * NC; e += blockDim.x) {
        const int r = e / NC, j = e - r * NC;
        const double2 v = M[r * 2 * NC + NC + j];
        inv[site * NC * NC + e] = make_float2((float)v.x, (float)v.y);
    }
}

// parity split / merge of coarse fields [V][64][n]: half p holds the sites of parity p, site s at s / 2
__global__ void k_parity_split(const float2 *__restrict__ full, float2 *__restrict__ he, float2 *__restrict__ ho,
                               TcArgs a) {
    const int64_t per = (int64_t)NC * a.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.V * per) return;
    const int64_t site = i / per, e = i - site * per;
    int c[4];
    site_to_coords(site, a.L, c);
    float2 *dst = ((c[0] + c[1] + c[2] + c[3]) & 1) ? ho : he;
    dst[(site >> 1) * per + e] = full[i];
}

__global__ void k_parity_merge_add(const float2 *__restrict__ he, const float2 *__restrict__ ho,
                                   float2 *__restrict__ full, TcArgs a) {
    const int64_t per = (int64_t)NC * a.n;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.V * per) return;
    const int64_t site = i / per, e = i - site * per;
    int c[4];
    site_to_coords(site, a.L, c);
    const float2 *src = ((c[0] + c[1] + c[2] + c[3]) & 1) ? ho : he;
    const float2 d = src[(site >> 1) * per + e];
    float2 z = full[i];
    z.x += d.x;
    z.y += d.y;
    full[i] = z;
}

}  // namespace

bool coarse_eo_supported(const Level &c) {
    if (!c.Abf.ptr) return false;
    for (int mu = 0; mu < 4; ++mu)
        if (c.L[mu] % 2) return false;
    return true;
}

void coarse_eo_prepare(Level &c, cudaStream_t s) {
    if (!coarse_eo_supported(c)) fail(MRHS_ERR_INVALID, "coarse even-odd needs 16-bit links and even coarse extents");
    DeviceBuffer inv(sizeof(float2) * (size_t)c.V * NC * NC);
    c.EoErr.alloc(sizeof(int));
    MRHS_CUDA(cudaMemsetAsync(c.EoErr.ptr, 0, sizeof(int), s));
    const size_t smem = sizeof(double2) * NC * 2 * NC;
    MRHS_CUDA(cudaFuncSetAttribute(k_self_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_self_inverse<<<(unsigned)c.V, 256, smem, s>>>(c.A32.as<float2>(), inv.as<float2>(), c.EoErr.as<int>());
    MRHS_LAUNCHED("k_self_inverse");
    c.AinvScale.alloc(sizeof(float) * (size_t)c.V);
    c.AinvBf.alloc((size_t)c.V * A_TILE);
    k_link_scale<<<(unsigned)c.V, 256, 0, s>>>(inv.as<float2>(), c.AinvScale.as<float>(), 1);
    MRHS_LAUNCHED("k_link_scale");
    const int64_t count = c.V * MROWS * NC;
    if (c.tc_fmt == MRHS_FP16)
        k_pack_links<0><<<ceil_div(count, 256), 256, 0, s>>>(inv.as<float2>(), c.AinvBf.as<uint8_t>(), c.V,
                                                             c.AinvScale.as<float>(), 1);
    else
        k_pack_links<1><<<ceil_div(count, 256), 256, 0, s>>>(inv.as<float2>(), c.AinvBf.as<uint8_t>(), c.V,
                                                             c.AinvScale.as<float>(), 1);
    MRHS_LAUNCHED("k_pack_links");
    int sing = 0;
    MRHS_CUDA(cudaMemcpyAsync(&sing, c.EoErr.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    MRHS_CUDA(cudaStreamSynchronize(s));
    if (sing) fail(MRHS_ERR_INVALID, "a coarse self block is singular: no coarse even-odd inverse");
}

void coarse_eo_hop(const Level &c, int out_parity, const float2 *in_half, float2 *out_half, const float2 *y_half,
                   int n, cudaStream_t s) {
    coarse_tc_general(c, c.Abf.as<uint8_t>() + A_TILE, c.LinkScale.as<float>(), 9, 1, 8, out_parity, in_half,
                      c.V / 2, out_half, y_half, n, s);
}

void coarse_eo_self(const Level &c, bool inverse, int parity, const float2 *in_half, float2 *out_half, int n,
                    cudaStream_t s) {
    if (inverse) {
        if (!c.AinvBf.ptr) fail(MRHS_ERR_INVALID, "coarse even-odd inverse not prepared");
        coarse_tc_general(c, c.AinvBf.as<uint8_t>(), c.AinvScale.as<float>(), 1, 0, 0, parity, in_half, c.V / 2,
                          out_half, nullptr, n, s);
    } else {
        coarse_tc_general(c, c.Abf.as<uint8_t>(), c.LinkScale.as<float>(), 9, 0, 0, parity, in_half, c.V / 2,
                          out_half, nullptr, n, s);
    }
}

void coarse_schur_apply(const Level &c, const float2 *in_o, float2 *out_o, float2 *tmp_e1, float2 *tmp_e2, int n,
                        cudaStream_t s) {
    // t = A_ee^-1 H_eo in_o;  out_o = A_oo in_o - H_oe t
    coarse_eo_hop(c, 0, in_o, tmp_e1, nullptr, n, s);
    coarse_eo_self(c, true, 0, tmp_e1, tmp_e2, n, s);
    coarse_eo_self(c, false, 1, in_o, out_o, n, s);
    coarse_eo_hop(c, 1, tmp_e2, out_o, out_o, n, s);
}

void coarse_parity_split(const Level &c, const float2 *full, float2 *he, float2 *ho, int n, cudaStream_t s) {
    TcArgs a{};
    for (int mu = 0; mu < 4; ++mu) a.L[mu] = c.L[mu];
    a.V = c.V;
    a.n = n;
    k_parity_split<<<ceil_div(c.V * NC * n, 256), 256, 0, s>>>(full, he, ho, a);
    MRHS_LAUNCHED("k_parity_split");
}

void coarse_parity_merge_add(const Level &c, const float2 *he, const float2 *ho, float2 *full, int n,
                             cudaStream_t s) {
    TcArgs a{};
    for (int mu = 0; mu < 4; ++mu) a.L[mu] = c.L[mu];
    a.V = c.V;
    a.n = n;
    k_parity_merge_add<<<ceil_div(c.V * NC * n, 256), 256, 0, s>>>(he, ho, full, a);
    MRHS_LAUNCHED("k_parity_merge_add");
}

int coarse_tc_error(const Level &c, cudaStream_t s) {
    if (!c.TcErr.ptr) return 0;
    int *e = pinned_flag_slot();
    read_back(e, c.TcErr.ptr, sizeof(int), s);
    MRHS_CUDA(cudaStreamSynchronize(s));
    return *e;
}

}  // namespace mrhs

extern "C" mrhs_status mrhs_debug_expire_waits(int launches) {
    if (launches < 0) return mrhs::api_record(MRHS_ERR_INVALID, "launches must be >= 0");
    mrhs::g_expire_waits.store(launches);
    return mrhs::api_record(MRHS_OK, "");
}
