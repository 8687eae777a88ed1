// TMA-staged step kernel (D3Q19, any storage format) for lattices whose x extent is a multiple
// of 64: the same site update as step_kernel (Eqs. 9-10, 34-35 with the boundary rules), with
// the streamed populations of the y/z-interior rows brought into shared memory by the Tensor
// Memory Accelerator instead of per-thread loads.
//
// A persistent block walks tiles of 64 x 4 sites (one z-plane) in x, y, z order.  Its loader
// warp issues, per tile, one cp.async.bulk.tensor box per population plane, shifted by -e_i so
// that the box holds exactly the sources of that plane's pulls (x-shifted planes load 72
// columns from an x start rounded down to 8, the rest 64), plus, for the 16-bit formats, the
// seven shifted windows of the FP32 temperature plane.  Loads run kStages tiles ahead and
// complete on a "full" mbarrier per stage; the eight compute warps release a stage through an
// "empty" mbarrier, so the bytes in flight no longer depend on the registers of the warps that
// compute and no barrier spans the block.  Warps whose sites are not y/z interior (boundary
// rows and planes, where the rules and the periodic wrap need other sources), and warps on a
// periodic x face, take the global-memory path of step_kernel; lanes on a walled or outflow x
// face apply the x-face rule of step_kernel after the staged loads.  The arithmetic and the
// values loaded are those of step_kernel: the results agree bit for bit.
//
// Every wait on an mbarrier is bounded by the global timer.  One that runs out sets an error
// flag and stops the warp; the loader then stops issuing and waits (bounded again) for the
// loads it has in flight before it leaves.  TmaGrid::extra_tx (zero in normal use) adds bytes
// to every stage's expected count that no load brings, so that a test can make the waits run
// out without any fault.
#define LBM_DEVICE_ONLY
#include "lbm_kernels.cu"

namespace lbm {
namespace {

constexpr int kTX = kTmaTileX, kTY = kTmaTileY;
constexpr int kTWarps = kTX * kTY / 32;     // compute warps of a block
constexpr int kTBlock = (kTWarps + 1) * 32;  // and one loader warp
constexpr unsigned long long kTmaWaitNs = 1000000000ull;  // 1 s per wait

template <class S>
struct TmaCfg {
    using T = typename S::T;
    static constexpr int kStages = sizeof(T) == 2 ? 3 : 2;
    static constexpr int kW = 72;  // slot width: 64 sites and 8 columns of halo
    static constexpr int kPlane = (kTY * kW * (int)sizeof(T) + 127) / 128 * 128;  // bytes
    static constexpr int kTSlot = S::kScaled ? (kTY * kW * 4 + 127) / 128 * 128 : 0;
    static constexpr int kStage = (kQ + kQT) * kPlane + kQT * kTSlot;
    static constexpr int kSmem = kStages * kStage + 128;  // + alignment of the base
};

// Stored value in shared memory as FP32.
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void bar_init_n(unsigned long long* b, unsigned n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}

__device__ __forceinline__ void bar_expect(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
                 "r"(bytes)
                 : "memory");
}
// True once the phase of the given parity has completed; false after kTmaWaitNs.
__device__ __forceinline__ bool bar_wait(unsigned long long* b, unsigned parity) {
    unsigned long long t0 = 0;
    while (true) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_addr(b)), "r"(parity)
            : "memory");
        if (done) return true;
        const unsigned long long t = now_ns();
        if (t0 == 0) t0 = t;
        else if (t - t0 > kTmaWaitNs) return false;
    }
}
__device__ __forceinline__ void tma4(void* dst, const CUtensorMap* map, int x, int y, int z, int q,
                                     unsigned long long* b) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(q), "r"(smem_addr(b))
        : "memory");
}
__device__ __forceinline__ void tma3(void* dst, const CUtensorMap* map, int x, int y, int z,
                                     unsigned long long* b) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(b))
        : "memory");
}

// Box of plane i (x start, width) for velocity component ex: the sources x - ex of 64 sites.
__device__ __forceinline__ int box_x(int x0, int ex) { return ex == 1 ? x0 - 8 : x0; }
// Column of site tx's source within the box.
__host__ __device__ constexpr int box_col(int ex) { return ex == 1 ? 7 : (ex == -1 ? 1 : 0); }

// Issue the loads of tile k into a stage (elected thread).
template <class S>
__device__ __forceinline__ void tma_issue(const KParams& p, const TmaGrid& tg, int k,
                                          unsigned char* stage, unsigned long long* b,
                                          const TmaMaps& m) {
    using C = TmaCfg<S>;
    using T = typename S::T;
    const int xt = k % tg.tiles_x, rest = k / tg.tiles_x;
    const int x0 = xt * kTX, y0 = (rest % tg.tiles_y) * kTY, z = rest / tg.tiles_y;
    unsigned bytes = 0;
#pragma unroll
    for (int i = 0; i < kQ; ++i) bytes += kTY * (ex19(i) ? 72 : 64) * (unsigned)sizeof(T);
#pragma unroll
    for (int j = 0; j < kQT; ++j)
        bytes += kTY * (ex7(j) ? 72 : 64) * (unsigned)(sizeof(T) + (S::kScaled ? 4 : 0));
    bar_expect(b, bytes + (unsigned)tg.extra_tx);
#pragma unroll
    for (int i = 0; i < kQ; ++i)
        tma4(stage + i * C::kPlane, ex19(i) ? &m.pop72 : &m.pop64, box_x(x0, ex19(i)),
             y0 - ey19(i), z - ez19(i), i, b);
#pragma unroll
    for (int j = 0; j < kQT; ++j)
        tma4(stage + (kQ + j) * C::kPlane, ex7(j) ? &m.pop72 : &m.pop64, box_x(x0, ex7(j)),
             y0 - ey7(j), z - ez7(j), kQ + j, b);
    if constexpr (S::kScaled) {
#pragma unroll
        for (int j = 0; j < kQT; ++j)
            tma3(stage + (kQ + kQT) * C::kPlane + j * C::kTSlot, ex7(j) ? &m.t72 : &m.t64,
                 box_x(x0, ex7(j)), y0 - ey7(j), z - ez7(j), b);
    }
}

// The site update of one thread from a staged tile (or from global memory, see the header).
template <bool HET, bool OUTF, class S>
__device__ __forceinline__ void tma_site(const KParams& p, const Planes& pl,
                                         const unsigned char* stage, int x, int y, int z, int tx,
                                         int r) {
    using C = TmaCfg<S>;
    using T = typename S::T;
    const bool valid = y < p.ny;  // x < nx: nx is a multiple of 64
    // staged boxes do not wrap: only rows strictly inside the y and z ranges use them; the
    // global-memory path takes the wider yz_fast set on its fast branch
    const bool yz_in = y > 0 && y < p.ny - 1 && z > 0 && z < p.nz - 1;
    const bool warp_yz_in = __all_sync(0xffffffffu, yz_in || !valid);
    const int mode = warp_gather_mode(p, x, y, z, valid);
    const unsigned lanes = __ballot_sync(0xffffffffu, valid);
    const bool xface = x == 0 || x == p.nx - 1;
    const bool periodic_x_face = (p.per_mask & 3u) && __any_sync(0xffffffffu, valid && xface);
    if (!valid) return;
    float f[kQ], g[kQT];
    const int s = x + p.nx * (y + p.ny * z);
    if (!warp_yz_in || periodic_x_face) {
        gather_site<OUTF, S, D3Q19>(pl, p, x, y, z, s, mode, f, g);
    } else {
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const T* src = reinterpret_cast<const T*>(stage + i * C::kPlane);
            f[i] = to_f32(src[r * (ex19(i) ? 72 : 64) + tx + box_col(ex19(i))]);
        }
#pragma unroll
        for (int j = 0; j < kQT; ++j) {
            const int at = r * (ex7(j) ? 72 : 64) + tx + box_col(ex7(j));
            const float v = to_f32(reinterpret_cast<const T*>(stage + (kQ + j) * C::kPlane)[at]);
            if constexpr (S::kScaled) {
                const float* tsrc = reinterpret_cast<const float*>(
                    stage + (kQ + kQT) * C::kPlane + j * C::kTSlot);
                g[j] = __fmul_rn(j == 0 ? p.om0 : p.om1, __fmaf_rn(p.sigma, tsrc[at], v));
            } else {
                g[j] = v;
            }
        }
        const int nxy = p.nx * p.ny;
        x_face_fixup<OUTF, S, D3Q19>(pl, p, x, y, z, s, lanes, x == 0, x == p.nx - 1, -p.nx, p.nx,
                                     -nxy, nxy, f, g);
    }
    finish_site<HET, OUTF, S, false, D3Q19>(pl, p, x, y, z, s, f, g);
}

// Warp roles: warps 0 .. 7 compute (warp w takes row w / 2, columns 32 (w % 2) .. + 31 of each
// tile), warp 8 loads.  Stage st of a block holds the tile of iteration it when it % kStages ==
// st; full[st] completes when its bytes have landed, empty[st] when the eight compute warps
// have read it.  No barrier spans the block, so compute warps drift apart by up to the
// pipeline depth instead of waiting for one another on every tile.
template <bool HET, bool OUTF, class S>
__global__ void __launch_bounds__(kTBlock, 3)
    tma_step_kernel(const __grid_constant__ KParams p, const __grid_constant__ Planes pl,
                    const __grid_constant__ TmaMaps m, const TmaGrid tg, int* __restrict__ err) {
    using C = TmaCfg<S>;
    constexpr int kS = C::kStages;
    extern __shared__ __align__(128) unsigned char sm_raw[];
    __shared__ __align__(8) unsigned long long full[kS], empty[kS];
    // stage slots start on 128-byte boundaries of the shared window
    unsigned char* sm = sm_raw + ((128u - (smem_addr(sm_raw) & 127u)) & 127u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < kS; ++i) {
            bar_init_n(&full[i], 1);
            bar_init_n(&empty[i], kTWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();  // the only block-wide barrier: barriers initialised
    dependent_launch_prologue();

    if (warp == kTWarps) {  // loader
        if (lane != 0) return;
        int it = 0;
        bool ok = true;
        for (int k = blockIdx.x; k < tg.ntiles; k += gridDim.x, ++it) {
            const int st = it % kS;
            if (it >= kS && !bar_wait(&empty[st], (unsigned)(it / kS - 1) & 1u)) {
                ok = false;  // a compute warp stopped: no further loads
                break;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_issue<S>(p, tg, k, sm + st * C::kStage, &full[st], m);
        }
        if (!ok) atomicExch(err, 1);
        // wait (bounded) for the loads still in flight before this thread leaves
        for (int j = it - kS > 0 ? it - kS : 0; j < it; ++j)
            if (!bar_wait(&full[j % kS], (unsigned)(j / kS) & 1u)) atomicExch(err, 1);
        return;
    }

    const int r = warp >> 1, tx = ((warp & 1) << 5) | lane;
    int it = 0;
    for (int k = blockIdx.x; k < tg.ntiles; k += gridDim.x, ++it) {
        const int st = it % kS;
        if (!__all_sync(0xffffffffu, bar_wait(&full[st], (unsigned)(it / kS) & 1u))) {
            if (lane == 0) atomicExch(err, 1);  // a load did not land in time: stop
            return;
        }
        const int xt = k % tg.tiles_x, rest = k / tg.tiles_x;
        const int x = xt * kTX + tx, y = (rest % tg.tiles_y) * kTY + r, z = rest / tg.tiles_y;
        tma_site<HET, OUTF, S>(p, pl, sm + st * C::kStage, x, y, z, tx, r);
        __syncwarp();
        if (lane == 0) bar_arrive(&empty[st]);  // this warp has read the stage
    }
}

template <bool HET, bool OUTF, class S>
const void* tma_fn() {
    return reinterpret_cast<const void*>(&tma_step_kernel<HET, OUTF, S>);
}

template <class S>
const void* tma_fn_of(bool het, bool outflow) {
    if (het && outflow) return tma_fn<true, true, S>();
    if (het) return tma_fn<true, false, S>();
    if (outflow) return tma_fn<false, true, S>();
    return tma_fn<false, false, S>();
}

}  // namespace

cudaError_t tma_prepare(const KParams& p, bool outflow, int* blocks, int* smem_bytes) {
    (void)outflow;
    return with_storage(p.storage, [&](auto tag) {
        using S = decltype(tag);
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        // all four variants (medium kind x outflow): the medium may change after selection
        int per_sm = 1 << 30;
        for (int v = 0; v < 4; ++v) {
            const void* fn = tma_fn_of<S>(v & 1, v & 2);
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     TmaCfg<S>::kSmem);
            if (e != cudaSuccess) return e;
            int n = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kTBlock, TmaCfg<S>::kSmem);
            if (e != cudaSuccess) return e;
            per_sm = n < per_sm ? n : per_sm;
        }
        *blocks = sms * per_sm;
        *smem_bytes = TmaCfg<S>::kSmem;
        return cudaSuccess;
    });
}

cudaError_t launch_step_tma(const KParams& p, bool outflow, const Planes& pl, const TmaMaps& m,
                            int blocks, int extra_tx, int* err, bool pdl, cudaStream_t st) {
    TmaGrid tg;
    tg.extra_tx = extra_tx;
    tg.tiles_x = p.nx / kTX;
    tg.tiles_y = (p.ny + kTY - 1) / kTY;
    tg.ntiles = tg.tiles_x * tg.tiles_y * p.nz;
    if (blocks > tg.ntiles) blocks = tg.ntiles;
    const bool het = p.phi_field != nullptr;
    return with_storage(p.storage, [&](auto tag) {
        using S = decltype(tag);
        auto k = het ? (outflow ? tma_step_kernel<true, true, S> : tma_step_kernel<true, false, S>)
                     : (outflow ? tma_step_kernel<false, true, S> : tma_step_kernel<false, false, S>);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(blocks);
        cfg.blockDim = dim3(kTBlock);
        cfg.dynamicSmemBytes = TmaCfg<S>::kSmem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = pdl ? 1 : 0;
        return cudaLaunchKernelEx(&cfg, k, p, pl, m, tg, err);
    });
}

}  // namespace lbm
