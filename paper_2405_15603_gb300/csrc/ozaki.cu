// FP64 matrix products on the BF16 tensor cores by error-free splitting.
//
// Ozaki, Ogita, Oishi and Rump (2012) split each operand into slices whose
// pairwise products are exact in the accumulator's precision; the product is
// the sum of the slice products.  Here, with a power-of-two scale per row of A
// (2^ea_i > max_k |A_ik|) and per column of B (2^eb_j):
//     A_ik = 2^ea_i (sum_{p=1..S} a_p[i,k] 2^{-pW} + r),   |r| < 2^{-SW},
// each slice a_p an integer in [-127, 127] (W = 7 bits, taken by truncation,
// so every slice and every remainder is exact in FP64), and likewise B.  A
// BF16 holds such an integer exactly, a product of two is below 2^14, and a
// sum of 1024 products below 2^24, so an FP32 tensor-core accumulation over a
// chunk of at most 1024 rows is exact.  Then
//     (A B)_ij ~ 2^{ea_i + eb_j} sum_{t=2..S+1} 2^{-tW} sum_{p+q=t} (a_p b_q)_ij,
// the products with p + q > S + 1 dropped (below K 2^{-(S+2)W} |A|_i |B|_j, with
// S = 8 at the level of FP64's own rounding).  The products of one level t
// share the scale 2^{-tW}, so they form ONE Gram contraction over the stacked
// slices: X = [a_1; ...; a_{t-1}] (A's slices transposed, (t-1)K x M) and
// Y = [b_{t-1}; ...; b_1] ((t-1)K x N); all levels of all the plan's products
// are the members of one grouped launch of the engine's Gram mode (row chunks
// of 1024 rows, FP32 partials per chunk).  The partials are integers, so their
// FP64 sums are exact; the levels are combined in FP64 from the smallest.
// B's slices are stored in reverse order, so that level t's Y is a contiguous
// tail of them.
#include <math.h>
#include <string.h>
#include <algorithm>

#include "ozaki.cuh"
#include "tc_engine.cuh"
#include "tc_kernels.cuh"

namespace {

constexpr int OZ_W = 7;                 // bits per slice
constexpr int OZ_S = 8;                 // slices per operand
constexpr int OZ_CHUNK = 1024;          // Gram rows per exact FP32 partial: 1024 * 127^2 < 2^24
constexpr double OZ_SLICE = 128.0;      // 2^W
static_assert(OZ_W * OZ_S == 56, "the slices cover the 56-bit fixed-point value");

struct OzDev {
    const double* A;
    const double* B;
    double* C;
    long long lda, ldb, ldc;
    int M, N, K, Mp, Np;
    int ta, tb;                         // A given as A^T (K x M), B as B^T (N x K)
    double alpha;
    __nv_bfloat16* X;                   // S blocks of K x Mp: slice p of A^T in block p - 1
    __nv_bfloat16* Y;                   // S blocks of K x Np: slice q of B in block S - q
    int* ea;                            // M
    int* eb;                            // N
    float* part[OZ_S];                  // level t = 2 + index: chunks x M x N
    int chunks[OZ_S];
};

// One operand's side of a product: the destination D[slice][r][c] (K x Cp
// blocks) holds the slices of V(r, c) 2^{-e_c}, where V(r, c) = src[c ld + r]
// (csrc: the source holds c along its rows) or src[r ld + c].
struct OzSide {
    const double* src;
    long long ld;
    int R, Cn, Cp;                      // R = K rows; Cn real and Cp padded columns
    int csrc;
    int reverse;                        // slice q in block S - q (B) instead of q - 1 (A)
    int* e;
    __nv_bfloat16* D;
};

__device__ __forceinline__ OzSide side_of(const OzDev& d, int which) {
    OzSide o;
    if (which == 0) {       // A: element (k, i) of A^T
        o.src = d.A; o.ld = d.lda; o.Cn = d.M; o.Cp = d.Mp; o.csrc = !d.ta; o.reverse = 0; o.e = d.ea; o.D = d.X;
    } else {                // B: element (k, j)
        o.src = d.B; o.ld = d.ldb; o.Cn = d.N; o.Cp = d.Np; o.csrc = d.tb; o.reverse = 1; o.e = d.eb; o.D = d.Y;
    }
    o.R = d.K;
    return o;
}

__device__ __forceinline__ double side_at(const OzSide& o, int r, int c) {
    return o.csrc ? o.src[(long long)c * o.ld + r] : o.src[(long long)r * o.ld + c];
}

__device__ __forceinline__ long long side_dst(const OzSide& o, int slice, int r, int c) {
    const int blk = o.reverse ? OZ_S - 1 - slice : slice;
    return ((long long)blk * o.R + r) * o.Cp + c;
}

// 2^e > |v| for the largest |v| (e = 0 for zeros).
__device__ __forceinline__ int exponent_above(double m) {
    int e = 0;
    if (m > 0.0) frexp(m, &e);
    return e;
}

// Column scales 2^e_c of every side: one warp per column where the column
// lies along the source's rows (8 columns per block), else 32 columns per
// block with 8 row groups each (coalesced along the source's rows);
// blockIdx.y = 2 g + side.
__global__ void __launch_bounds__(256) k_oz_exponents(const OzDev* g) {
    const OzSide o = side_of(g[blockIdx.y / 2], blockIdx.y % 2);
    __shared__ double red[8][33];
    double m = 0.0;
    if (o.csrc) {
        const int c = blockIdx.x * 8 + threadIdx.x / 32, lane = threadIdx.x % 32;
        if (c >= o.Cn) return;
        for (int r = lane; r < o.R; r += 32) m = fmax(m, fabs(o.src[(long long)c * o.ld + r]));
        for (int w = 16; w > 0; w >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, w));
        if (lane == 0) o.e[c] = exponent_above(m);
        return;
    }
    if (blockIdx.x * 32 >= (unsigned)o.Cn) return;         // uniform over the block
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32, c = blockIdx.x * 32 + tx;
    if (c < o.Cn)
        for (int r = ty; r < o.R; r += 8) m = fmax(m, fabs(o.src[(long long)r * o.ld + c]));
    red[ty][tx] = m;
    __syncthreads();
    if (ty == 0 && c < o.Cn) {
        for (int k = 1; k < 8; k++) m = fmax(m, red[k][tx]);
        o.e[c] = exponent_above(m);
    }
}

// The slicing of one value: v 2^{56 - e} truncated to an integer (|.| < 2^56,
// exact in int64) whose 7-bit groups, from the top, are the slices' magnitudes
// (the same values as repeated truncation of v 2^{-e} in FP64, taken with
// integer operations).
__device__ __forceinline__ long long oz_fixed(double v, int e) { return (long long)ldexp(v, 56 - e); }

__device__ __forceinline__ float oz_digit(long long m, int q) {
    const long long u = m < 0 ? -m : m;
    const int d = (int)((u >> (49 - OZ_W * q)) & 127);
    return (float)(m < 0 ? -d : d);
}

// Slices of a side whose source is laid out like the destination: one
// thread per element, along c.
__global__ void __launch_bounds__(256) k_oz_slice_direct(const OzDev* g) {
    const OzSide o = side_of(g[blockIdx.z / 2], blockIdx.z % 2);
    if (o.csrc) return;
    const int c = blockIdx.x * 256 + threadIdx.x, r = blockIdx.y;
    if (c >= o.Cp || r >= o.R) return;
    const long long m = (c < o.Cn) ? oz_fixed(side_at(o, r, c), o.e[c]) : 0;
#pragma unroll
    for (int q = 0; q < OZ_S; q++) o.D[side_dst(o, q, r, c)] = __float2bfloat16_rn(oz_digit(m, q));
}

// Slices of a side whose source holds c along its rows: a 32 x 32 tile
// through shared memory, read along r and written along c.
__global__ void __launch_bounds__(256) k_oz_slice_transpose(const OzDev* g) {
    const OzSide o = side_of(g[blockIdx.z / 2], blockIdx.z % 2);
    if (!o.csrc) return;
    const int c0 = blockIdx.y * 32, r0 = blockIdx.x * 32;
    if (c0 >= o.Cp || r0 >= o.R) return;
    __shared__ long long x[32][33];
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
    for (int cc = ty; cc < 32; cc += 8) {       // read along r (tx)
        const int c = c0 + cc, r = r0 + tx;
        x[cc][tx] = (c < o.Cn && r < o.R) ? oz_fixed(side_at(o, r, c), o.e[c]) : 0;
    }
    __syncthreads();
    for (int rr = ty; rr < 32; rr += 8) {       // write along c (tx)
        const int r = r0 + rr, c = c0 + tx;
        if (r >= o.R || c >= o.Cp) continue;
        const long long m = x[tx][rr];
#pragma unroll
        for (int q = 0; q < OZ_S; q++) o.D[side_dst(o, q, r, c)] = __float2bfloat16_rn(oz_digit(m, q));
    }
}

// C = 2^{ea_i + eb_j} sum_t 2^{-tW} S_t, S_t the integer sum of level t's
// exact partials (integer adds), the levels by Horner's rule from the
// smallest (each step one exact scaling and one rounding FP64 add).
__global__ void __launch_bounds__(256) k_oz_combine(const OzDev* g) {
    const OzDev d = g[blockIdx.y];
    const long long e = (long long)blockIdx.x * 256 + threadIdx.x;
    if (e >= (long long)d.M * d.N) return;
    const int i = (int)(e / d.N), j = (int)(e % d.N);
    const long long mn = (long long)d.M * d.N;
    double acc = 0.0;
    for (int l = OZ_S - 1; l >= 0; l--) {
        long long sl = 0;
        for (int c = 0; c < d.chunks[l]; c++) sl += (long long)__float2int_rn(d.part[l][c * mn + e]);
        acc = fma(acc, 1.0 / OZ_SLICE, (double)sl);
    }
    d.C[(long long)i * d.ldc + j] = d.alpha * ldexp(acc, d.ea[i] + d.eb[j] - 2 * OZ_W);
}

int round_up_i(int a, int b) { return (a + b - 1) / b * b; }

}  // namespace

struct OzPlan {
    int n;                               // products
    int maxM, maxN, maxK, maxMp, maxNp;
    long long maxMN;
    OzDev* dev;                          // n descriptors
    void* ws;                            // slices, exponents and partials
    unsigned char* tabs;                 // the member table: Args, start blocks, grids
    GroupTab tab;                        // every (product, level) of the grouped Gram launch
    unsigned blocks;
};

kfac_status_t oz_plan_create(const std::vector<OzGemm>& gemms, int* status, OzPlan** out) {
    *out = nullptr;
    if (gemms.empty()) return KFAC_BAD_ARG;
    OzPlan* p = new OzPlan();
    memset(p, 0, sizeof(*p));
    *out = p;
    p->n = (int)gemms.size();
    std::vector<OzDev> hd(p->n);
    size_t bytes = 0;
    auto take = [&](size_t sz) {
        bytes = (bytes + 255) / 256 * 256;
        const size_t at = bytes;
        bytes += sz;
        return at;
    };
    struct Off {
        size_t X, Y, ea, eb, part[OZ_S];
    };
    std::vector<Off> off(p->n);
    for (int g = 0; g < p->n; g++) {
        const OzGemm& G = gemms[g];
        if (G.M < 1 || G.N < 1 || G.K < 1 || G.K > OZ_MAX_K) return KFAC_BAD_ARG;
        OzDev& d = hd[g];
        memset(&d, 0, sizeof(d));
        d.A = G.A; d.B = G.B; d.C = G.C;
        d.lda = G.lda; d.ldb = G.ldb; d.ldc = G.ldc;
        d.M = G.M; d.N = G.N; d.K = G.K;
        d.alpha = G.alpha;
        d.ta = G.ta ? 1 : 0;
        d.tb = G.tb ? 1 : 0;
        d.Mp = round_up_i(G.M, 64);
        d.Np = round_up_i(G.N, 64);
        off[g].X = take(sizeof(__nv_bfloat16) * (size_t)OZ_S * G.K * d.Mp);
        off[g].Y = take(sizeof(__nv_bfloat16) * (size_t)OZ_S * G.K * d.Np);
        off[g].ea = take(sizeof(int) * (size_t)G.M);
        off[g].eb = take(sizeof(int) * (size_t)G.N);
        for (int l = 0; l < OZ_S; l++) {
            const int rows = (l + 1) * G.K;
            d.chunks[l] = (rows + OZ_CHUNK - 1) / OZ_CHUNK;
            off[g].part[l] = take(sizeof(float) * (size_t)d.chunks[l] * G.M * G.N);
        }
        p->maxM = std::max(p->maxM, G.M);
        p->maxN = std::max(p->maxN, G.N);
        p->maxK = std::max(p->maxK, G.K);
        p->maxMp = std::max(p->maxMp, d.Mp);
        p->maxNp = std::max(p->maxNp, d.Np);
        p->maxMN = std::max(p->maxMN, (long long)G.M * G.N);
    }
    kfac_status_t st;
    if ((st = kfac_device_alloc(&p->ws, bytes))) return st;
    unsigned char* base = (unsigned char*)p->ws;
    for (int g = 0; g < p->n; g++) {
        OzDev& d = hd[g];
        d.X = (__nv_bfloat16*)(base + off[g].X);
        d.Y = (__nv_bfloat16*)(base + off[g].Y);
        d.ea = (int*)(base + off[g].ea);
        d.eb = (int*)(base + off[g].eb);
        for (int l = 0; l < OZ_S; l++) d.part[l] = (float*)(base + off[g].part[l]);
    }
    void* dv = nullptr;
    if ((st = kfac_device_alloc(&dv, sizeof(OzDev) * p->n))) return st;
    p->dev = (OzDev*)dv;
    if (cudaMemcpy(p->dev, hd.data(), sizeof(OzDev) * p->n, cudaMemcpyHostToDevice) != cudaSuccess)
        return KFAC_CUDA_ERROR;

    // the member table of the grouped Gram launch: every (product, level),
    // the members with the most blocks first
    using GC = tck::Cfg<tck::GRAM>;
    const size_t stride = (sizeof(tck::Args) + 63) / 64 * 64;
    const int nm = p->n * OZ_S;
    struct Mem {
        int g, l;
        unsigned blocks;
    };
    std::vector<Mem> mem;
    for (int g = 0; g < p->n; g++) {
        const OzDev& d = hd[g];
        const int tiles = ((d.M + tck::BM - 1) / tck::BM) * ((d.N + GC::BN - 1) / GC::BN);
        for (int l = 0; l < OZ_S; l++) mem.push_back(Mem{g, l, (unsigned)(tiles * d.chunks[l])});
    }
    std::stable_sort(mem.begin(), mem.end(), [](const Mem& x, const Mem& y) { return x.blocks > y.blocks; });
    const size_t start_off = stride * nm;
    const size_t grid_off = start_off + (sizeof(unsigned) * nm + 15) / 16 * 16;
    std::vector<unsigned char> host(grid_off + sizeof(uint3) * nm + 16, 0);
    void* tv = nullptr;
    if ((st = kfac_device_alloc(&tv, host.size()))) return st;
    p->tabs = (unsigned char*)tv;
    unsigned long long blocks = 0;
    for (int m = 0; m < nm; m++) {
        const OzDev& d = hd[mem[m].g];
        const int l = mem[m].l, t = l + 2;
        tck::Args a;
        memset(&a, 0, sizeof(a));
        const int rows = (t - 1) * d.K;
        const __nv_bfloat16* ybase = d.Y + (size_t)(OZ_S - t + 1) * d.K * d.Np;
        if (!tc_make_tmap_2d(&a.a0, d.X, d.Mp, rows, (uint64_t)d.Mp * 2, 64, 64) ||
            !tc_make_tmap_2d(&a.b0, ybase, d.Np, rows, (uint64_t)d.Np * 2, 64, 64))
            return KFAC_CUDA_ERROR;
        a.P = d.M;
        a.Q = d.N;
        a.rows = rows;
        a.row_chunk = OZ_CHUNK;
        a.sym = 0;
        a.q_tiles = (d.N + GC::BN - 1) / GC::BN;
        a.part = d.part[l];
        a.status = status;
        const int tiles = ((d.M + tck::BM - 1) / tck::BM) * a.q_tiles;
        const uint3 grid = make_uint3(tiles, d.chunks[l], 1);
        const unsigned b0 = (unsigned)blocks;
        memcpy(host.data() + stride * m, &a, sizeof(a));
        memcpy(host.data() + start_off + sizeof(unsigned) * m, &b0, sizeof(unsigned));
        memcpy(host.data() + grid_off + sizeof(uint3) * m, &grid, sizeof(uint3));
        blocks += (unsigned long long)tiles * d.chunks[l];
    }
    if (blocks >= (1ull << 31)) return KFAC_BAD_ARG;
    p->tab.packs = p->tabs;
    p->tab.start = (const unsigned*)(p->tabs + start_off);
    p->tab.grid = (const uint3*)(p->tabs + grid_off);
    p->tab.n = nm;
    p->tab.stride = (int)stride;
    p->blocks = (unsigned)blocks;
    if (cudaMemcpy(p->tabs, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return KFAC_CUDA_ERROR;
    return KFAC_OK;
}

kfac_status_t oz_run(kfac_pinn_handle* h, OzPlan* p, cudaStream_t s) {
    const int n = p->n;
    const int maxC = std::max(p->maxMp, p->maxNp);
    k_oz_exponents<<<dim3(ceil_div_u(maxC, 8), 2 * n), 256, 0, s>>>(p->dev);
    KFAC_LAUNCH_CHECK(h);
    k_oz_slice_direct<<<dim3(ceil_div_u(maxC, 256), p->maxK, 2 * n), 256, 0, s>>>(p->dev);
    KFAC_LAUNCH_CHECK(h);
    k_oz_slice_transpose<<<dim3(ceil_div_u(p->maxK, 32), ceil_div_u(maxC, 32), 2 * n), 256, 0, s>>>(p->dev);
    KFAC_LAUNCH_CHECK(h);
    const cudaError_t e = tck::engine_group_launcher(tck::GRAM, false)(p->tab, p->blocks, 0, s);
    if (e != cudaSuccess) {
        kfac_record_cuda_error(e);
        return KFAC_CUDA_ERROR;
    }
    h->launches++;
    k_oz_combine<<<dim3(ceil_div_u(p->maxMN, 256), n), 256, 0, s>>>(p->dev);
    KFAC_LAUNCH_CHECK(h);
    return KFAC_OK;
}

void oz_plan_free(OzPlan* p) {
    if (!p) return;
    cudaFree(p->ws);
    cudaFree(p->dev);
    cudaFree(p->tabs);
    delete p;
}
