// sl1m_noalloc.cu -- sl1m_forward_noalloc: the forward operator for callers
// that must not allocate device memory at the time of the call.
//
// Some callers cannot call cudaMalloc when they need the operator: a process
// whose device memory is handed out by a pool or by another framework that
// does not let libraries grow their own, or a latency-critical loop that must
// never enter the allocator (cudaMalloc/cudaFree can synchronise the device).
// This entry point keeps every byte of scratch the forward path needs -- the
// problem descriptor, the work-split tables, the input in the library's
// pixel order, the stream-K partial sums and the output before it is put back
// in the caller's order -- in one file-scope __device__ array of fixed size,
// SCRATCH_BYTES, that every GPU loading this library holds until the process
// exits.  The call makes no cudaMalloc / cudaFree and calls no allocating
// library routine.  The paper has no counterpart: this is plumbing.
//
// The per-call host data (descriptor, plan header and work-split tables) is
// built on the host and written into the array by small kernels that carry
// it in their parameters: a launch snapshots its parameters, so the call
// enqueues work and returns without waiting for the stream (a copy from
// pageable host memory would wait for it), and the host data may go out of
// scope at once.
#include <cstring>
#include <mutex>
#include <vector>

#include "sl1m_host.h"
#include "sl1m_kernels.h"

using namespace sl1m;

namespace {

constexpr size_t SCRATCH_BYTES = (size_t)32 << 20;   // 32 MiB
constexpr int MAX_DEVICES = 64;

__device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// Device address of g_scratch, resolved once per device (host code may not
// use the symbol itself: on the host it names a stand-in, not device memory).
void* g_scratch_dev[MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mu;

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Up to STAGE_WORDS 32-bit words of host data, carried by value in a kernel's
// parameters (16 KB, inside the 32 KB parameter space of sm_70 and later).
constexpr int STAGE_WORDS = 4096;
struct StageChunk {
    unsigned* dst;
    int n_words;
    unsigned w[STAGE_WORDS];
};

__global__ void __launch_bounds__(256) stage_words_kernel(const StageChunk c)
{
    for (int i = threadIdx.x; i < c.n_words; i += blockDim.x) c.dst[i] = c.w[i];
}

// Write n_bytes (a multiple of 4) of host data to dst on stream st, in
// chunks of STAGE_WORDS words; returns the launches made through *n_launch.
cudaError_t stage_to_device(unsigned char* dst, const unsigned char* src, size_t n_bytes, cudaStream_t st,
                            long long* n_launch)
{
    StageChunk c;
    for (size_t at = 0; at < n_bytes; at += sizeof(c.w)) {
        const size_t nb = std::min(sizeof(c.w), n_bytes - at);
        c.dst = (unsigned*)(dst + at);
        c.n_words = (int)(nb / 4);
        std::memcpy(c.w, src + at, nb);
        stage_words_kernel<<<1, 256, 0, st>>>(c);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        ++*n_launch;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" int sl1m_forward_noalloc(sl1m_problem* prob, const double* x_dev, double* vis_out_dev, int precision)
{
    if (!prob) return SL1M_ERR_ARG;
    sl1m_ctx* ctx = prob->ctx;
    if (ctx->server) return sl1m_fail(ctx, SL1M_ERR_BUSY, "a server is running on this context");
    if (!x_dev || !vis_out_dev) return sl1m_fail(ctx, SL1M_ERR_ARG, "null pointer");
    if (precision != SL1M_FP64 && precision != SL1M_MIXED)
        return sl1m_fail(ctx, SL1M_ERR_ARG, "precision must be SL1M_FP64 or SL1M_MIXED");
    if (prob->dirty || !prob->dev)
        return sl1m_fail(ctx, SL1M_ERR_STATE,
                         "problem not laid out on the device yet: call any allocating operator call "
                         "(e.g. sl1m_forward) once after setting its inputs");
    if (ctx->device < 0 || ctx->device >= MAX_DEVICES) return sl1m_fail(ctx, SL1M_ERR_ARG, "device index too large");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return sl1m_fail(ctx, SL1M_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    // set-up, once per device, with that device current
    unsigned char* base;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_dev[ctx->device]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess || !ptr)
                return sl1m_fail(ctx, SL1M_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
            g_scratch_dev[ctx->device] = ptr;
        }
        base = (unsigned char*)g_scratch_dev[ctx->device];
    }
    const DevProblem& lay = prob->hp;
    const bool gains = prob->n_ant > 0;
    // work split of this single problem (host tables)
    HostPlan H;
    const int which = precision == SL1M_FP64 ? 0 : 2;
    plan_host({lay.vis.n_blk}, {lay.pix.n_gran}, ctx->num_sms * occupancy(which, gains, std::max(1, prob->n_ant)), H);
    // carve the static scratch
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off += align256(bytes);
        return base + at;
    };
    DevProblem* d_desc = (DevProblem*)take(sizeof(DevProblem));
    Plan* d_plan = (Plan*)take(sizeof(Plan));
    long long* d_u0 = (long long*)take(sizeof(long long) * H.u0.size());
    int* d_b0 = (int*)take(sizeof(int) * H.b0.size());
    int* d_poff = (int*)take(sizeof(int) * std::max<size_t>(1, H.poff.size()));
    int* d_clo = (int*)take(sizeof(int) * std::max<size_t>(1, H.clo.size()));
    int* d_ncon = (int*)take(sizeof(int) * std::max<size_t>(1, H.ncon.size()));
    double* d_x = (double*)take(sizeof(double) * lay.pix.n_pad);
    double2* d_out = (double2*)take(sizeof(double2) * lay.vis.n_pad);
    double2* d_part = (double2*)take(sizeof(double2) * (size_t)std::max(1, H.n_slots) * BLK);
    if (off > SCRATCH_BYTES)
        return sl1m_fail(ctx, SL1M_ERR_ARG,
                         "problem needs %zu bytes of scratch; sl1m_forward_noalloc holds %zu (32 MiB)", off,
                         SCRATCH_BYTES);
    // descriptor, plan header and tables: laid out on the host exactly as the
    // scratch is carved above, then written by kernels carrying them by value
    DevProblem d = lay;
    d.st = nullptr;
    d.x = d_x;
    d.r = nullptr;
    d.fwd_out = d_out;
    d.adj_out = nullptr;
    Plan pl{};
    pl.n_probs = 1;
    pl.C = H.C;
    pl.U = H.U;
    pl.prob_u0 = d_u0;
    pl.prob_b0 = d_b0;
    pl.blk_poff = d_poff;
    pl.blk_clo = d_clo;
    pl.blk_ncon = d_ncon;
    pl.n_blocks = H.n_blocks;
    pl.n_slots = H.n_slots;
    const size_t head = (size_t)((unsigned char*)d_x - base);     // descriptor .. tables
    std::vector<unsigned char> img(head, 0);
    auto put = [&](void* at, const void* src, size_t bytes) {
        if (bytes) std::memcpy(img.data() + ((unsigned char*)at - base), src, bytes);
    };
    const int zero = 0;
    put(d_desc, &d, sizeof d);
    put(d_plan, &pl, sizeof pl);
    put(d_u0, H.u0.data(), sizeof(long long) * H.u0.size());
    put(d_b0, H.b0.data(), sizeof(int) * H.b0.size());
    if (!H.poff.empty()) {
        put(d_poff, H.poff.data(), sizeof(int) * H.poff.size());
        put(d_clo, H.clo.data(), sizeof(int) * H.clo.size());
        put(d_ncon, H.ncon.data(), sizeof(int) * H.ncon.size());
    } else {
        put(d_ncon, &zero, sizeof(int));
    }
    cudaStream_t st = ctx->stream;
#define CKN(call)                                                                                     \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return sl1m_fail(ctx, SL1M_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)
    CKN(stage_to_device(base, img.data(), head, st, &ctx->n_launch));
    // every partial slot the finish reads is written by exactly one CTA of this
    // launch, so nothing in the scratch needs clearing
    CKN(launch_gather_real(x_dev, d_x, lay.pix.orig, lay.pix.n_pad, 1.0, st));
    CKN(launch_forward(precision == SL1M_FP64 ? 0 : 1, gains, prob->n_ant, d_desc, d_plan, H.C, d_part, st));
    CKN(launch_fwd_finish(d_desc, d_plan, std::max(1, std::min(H.n_blocks, 4 * ctx->num_sms)), d_part, st));
    CKN(launch_scatter_cplx(d_out, (double2*)vis_out_dev, lay.vis.orig, lay.vis.n_pad, st));
#undef CKN
    ctx->n_launch += 4;
    return SL1M_OK;
}
