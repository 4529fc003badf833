// K(w) x for callers that cannot allocate device memory (pbm_apply_K_noalloc).
//
// Some callers of this library cannot call cudaMalloc: real-time loops that must not allocate after
// start-up, host frameworks whose own allocator owns every byte of device memory, and plug-ins that
// run inside such hosts. They cannot create a grid handle, because pbm_create_grid allocates its
// hierarchy and workspace. This file gives them the FP64 fine-level apply y = K(w) x of pbm_apply_K
// without a handle: the caller passes the grid description and its own input and output arrays, and
// the scratch that the two column passes need (plane quads, per-CTA partial sums, the last-CTA
// counter) lives in one file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.
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

// partial sums of the node pass: two per CTA, at most kNodeBlocksPerSm CTAs per SM
static size_t noalloc_partials(int sms) { return size_t(2) * size_t(sms) * kNodeBlocksPerSm; }

// bytes of scratch an apply on grid G needs (scalar block, partial sums, plane quads); G has passed
// the 32-bit index check, so the int64 products below cannot wrap
static size_t noalloc_bytes(const Geom& G, int sms) {
    return align_up(sizeof(DevScalars)) + align_up(sizeof(double) * noalloc_partials(sms)) +
           sizeof(double) * size_t(cols_scratch_entries(G));
}

// the device a caller's array lives on (host-only query); PBM_EINVAL for memory the CUDA runtime
// does not know or that is on another device than the current one
static void check_on_device(const void* p, int dev, const char* name) {
    cudaPointerAttributes at{};
    const cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        fail(PBM_EINVAL, std::string(name) + ": not a pointer the CUDA runtime knows");
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        fail(PBM_EINVAL, std::string(name) + " must be device memory");
    if (at.type == cudaMemoryTypeDevice && at.device != dev)
        fail(PBM_EINVAL, std::string(name) + " is on device " + std::to_string(at.device) +
                             ", the current device is " + std::to_string(dev));
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
        // sizes in double first, so that no integer expression below can wrap (the same 32-bit index
        // limit as pbm_create_grid)
        if (3.0 * (nx + 1.0) * (ny + 1.0) * (nz + 1.0) >= 2147483647.0 || 8.0 * double(nx) * ny * nz >= 2147483647.0)
            fail(PBM_EINVAL, "grid too large for pbm_apply_K_noalloc: the kernels index nodes and elements with "
                             "32-bit integers");
        const Geom G{nx, ny, nz, support};
        int dev = 0;
        PBM_CUDA(cudaGetDevice(&dev));
        const int sms = num_sms();
        const size_t need = noalloc_bytes(G, sms);
        if (need > NOALLOC_SCRATCH_BYTES)
            fail(PBM_EINVAL, "grid too large for pbm_apply_K_noalloc: it needs " + std::to_string(need) +
                                 " bytes of scratch, the static array holds " +
                                 std::to_string(NOALLOC_SCRATCH_BYTES) + " (grids of up to about 170,000 elements always fit)");
        check_on_device(w_dev, dev, "w");
        check_on_device(x_dev, dev, "x");
        check_on_device(y_dev, dev, "y");
        unsigned char* base = noalloc_scratch(dev);
        const cudaStream_t st = (cudaStream_t)stream;
        ColEnv env;
        env.sc = (DevScalars*)base;
        env.partials = (double*)(base + align_up(sizeof(DevScalars)));
        env.partials_len = int64_t(noalloc_partials(sms));
        double* quads = (double*)(base + align_up(sizeof(DevScalars)) + align_up(sizeof(double) * noalloc_partials(sms)));
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
