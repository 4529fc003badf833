// K(w) x for callers that cannot allocate device memory (pbm_apply_K_noalloc).
//
// Some callers of this library cannot call cudaMalloc: code that runs while a CUDA graph is being
// captured (allocation is not a capturable operation), real-time loops that must not allocate after
// start-up, and host frameworks whose own allocator owns every byte of device memory. They cannot
// create a grid handle, because pbm_create_grid allocates its hierarchy and workspace. This file
// gives them the FP64 fine-level apply y = K(w) x of pbm_apply_K without a handle: the caller
// passes the grid description and its own input and output arrays, and the scratch that the two
// column passes need (plane quads, per-CTA partial sums, the last-CTA counter) lives in one
// file-scope device array of fixed size, which every GPU that loads the library holds until the
// process exits.
#include <mutex>

#include "pbm_internal.h"

namespace pbm {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;   // 32 MiB per device
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// The array's name in host code is only a host-side stand-in for the symbol. Its device address is
// looked up once per device (with that device current) and cached; kernels get that address.
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

static unsigned char* noalloc_scratch(int device) {
    if (device < 0 || device >= NOALLOC_MAX_DEVICES) fail(PBM_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            fail(PBM_ECUDA, std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
        g_noalloc_ptr[device] = p;
    }
    return (unsigned char*)g_noalloc_ptr[device];
}

static size_t align_up(size_t v) { return (v + 255) / 256 * 256; }

// bytes of scratch an apply on grid G needs (scalar block, partial sums, plane quads)
static size_t noalloc_bytes(const Geom& G) {
    return align_up(sizeof(DevScalars)) + align_up(sizeof(double) * 2 * 152 * 8) +
           sizeof(double) * size_t(cols_scratch_entries(G));
}

}  // namespace pbm

using namespace pbm;

extern "C" int pbm_apply_K_noalloc(int nx, int ny, int nz, int support, double E, double nu, double h,
                                   const double* w_dev, const double* x_dev, double* y_dev, void* stream) {
    try {
        if (!w_dev || !x_dev || !y_dev) fail(PBM_EINVAL, "null argument");
        if (nx < 1 || ny < 1 || nz < 1) fail(PBM_EINVAL, "grid dimensions must be >= 1");
        if (support < PBM_CANTILEVER || support > PBM_FREE) fail(PBM_EINVAL, "unknown support");
        if (!(E > 0.0) || !(nu > -1.0 && nu < 0.5) || !(h > 0.0)) fail(PBM_EINVAL, "bad material or h");
        const Geom G{nx, ny, nz, support};
        const size_t need = noalloc_bytes(G);
        if (need > NOALLOC_SCRATCH_BYTES)
            fail(PBM_EINVAL, "grid too large for pbm_apply_K_noalloc: it needs " + std::to_string(need) +
                                 " bytes of scratch, the static array holds " +
                                 std::to_string(NOALLOC_SCRATCH_BYTES) + " (about 170,000 elements)");
        int dev = 0;
        PBM_CUDA(cudaGetDevice(&dev));
        unsigned char* base = noalloc_scratch(dev);
        const cudaStream_t st = (cudaStream_t)stream;
        ColEnv env;
        env.sc = (DevScalars*)base;
        env.partials = (double*)(base + align_up(sizeof(DevScalars)));
        env.partials_len = 2 * 152 * 8;
        double* quads = (double*)(base + align_up(sizeof(DevScalars)) + align_up(sizeof(double) * 2 * 152 * 8));
        env.qa = quads;
        env.qb = quads + 12 * int64_t(nx) * ny * (nz + 1);
        // the last-CTA counter must start at zero (a previous call leaves it at zero, an aborted one
        // might not)
        PBM_CUDA(cudaMemsetAsync(&env.sc->counter[0], 0, sizeof(unsigned int), st));
        KeHat kh;
        element_hat(E, nu, h, kh);
        ApplyArgs a{};
        a.x = x_dev;
        a.y = y_dev;
        a.mode = EPI_APPLY;
        a.dot_slot = -1;
        cols_fine_env<double>(env, G, kh, w_dev, nullptr, nullptr, nullptr, a, st);
    } catch (const Error& e) {
        set_error(e.msg);
        return e.code;
    }
    set_error("");
    return PBM_OK;
}
