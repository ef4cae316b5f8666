// poisson_vcycle_noalloc: one multigrid V-cycle without a plan and without allocating.
//
// Some callers cannot call cudaMalloc: code running under another framework's memory
// manager that has reserved the device memory, or a latency-critical loop that cannot
// afford the implicit device synchronisation of cudaMalloc / cudaFree.  For them the
// library keeps one statically sized device array (NOALLOC_BYTES below) holding the
// instance descriptor, its state, the work items and the multigrid level arrays; the
// caller still provides the right-hand side and the iterate.  The same kernels as
// poisson_vcycle run on it, so both entry points give the same cycle.
//
// In host code the array's name is only a host-side stand-in, never a device address:
// the first call on each device (with that device current) asks the runtime for the
// array's device address with cudaGetSymbolAddress and caches it; that first call also
// raises the kernels' shared-memory limits, and should therefore come before any stream
// capture.  Every call reuses the same array and clears the part it uses; calls that
// overlap on the GPU (two streams, two host threads) race on it.
//
// Nothing is copied from host memory: the descriptor, state and work items travel as a
// kernel argument to a one-block kernel that writes them into the array, so a call only
// enqueues work and returns without waiting for the stream.
#include "../../include/helm.h"
#include "launch.h"

#include <cstring>
#include <mutex>

namespace {

using namespace helm;

constexpr size_t NOALLOC_BYTES = (size_t)16 << 20;   // 16 MiB per device, held until exit
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_scratch[NOALLOC_BYTES];

struct DeviceScratch {
    unsigned char* ptr = nullptr;
    bool ready = false;
};
DeviceScratch g_dev[MAX_DEVICES];
std::mutex g_mu;

constexpr size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// layout of the array: descriptor | state | work items | level arrays
constexpr size_t OFF_STATE = a256(sizeof(InstDesc));
constexpr size_t OFF_ITEMS = OFF_STATE + a256(sizeof(InstState));
constexpr size_t OFF_LEVELS = OFF_ITEMS + a256(sizeof(MgItem) * HELM_MAXLEV);

inline helm_status fail(helm_status st, const char*) { return st; }

// The array's header (descriptor | state | work items) as one kernel argument.
struct alignas(16) Header {
    unsigned char bytes[OFF_LEVELS];
};
static_assert(sizeof(Header) <= 4096, "header must fit the kernel-argument space");

__global__ void k_noalloc_header(Header hd, unsigned char* dst)
{
    const unsigned int* src = reinterpret_cast<const unsigned int*>(hd.bytes);
    unsigned int* out = reinterpret_cast<unsigned int*>(dst);
    for (int i = threadIdx.x; i < (int)(OFF_LEVELS / 4); i += blockDim.x) out[i] = src[i];
}

helm_status device_scratch(unsigned char** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return fail(HELM_ECUDA, "no usable current device");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev[dev].ready) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return fail(HELM_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
        }
        for (int D = 2; D <= 3; ++D)
            for (int prec = 0; prec <= 1; ++prec)
                if (setup_tail(D, prec) != cudaSuccess) return fail(HELM_ECUDA, "kernel set-up failed");
        if (setup_2d(0) != cudaSuccess || setup_2d(1) != cudaSuccess)
            return fail(HELM_ECUDA, "kernel set-up failed");
        g_dev[dev].ptr = (unsigned char*)p;
        g_dev[dev].ready = true;
    }
    *out = g_dev[dev].ptr;
    return HELM_OK;
}

// A 16-byte aligned pointer to managed memory or to memory of the current device (the
// kernels and the scratch array live on the current device; another GPU's memory would
// need peer access the library does not set up).
bool device_ptr(const void* p)
{
    if (!p || ((uintptr_t)p & 15) != 0) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" helm_status poisson_vcycle_noalloc(int ndim, int n, double h, int prec, const void* rhs,
                                              void* e, int nu1, int nu2, void* cuda_stream)
{
    if (ndim != 2 && ndim != 3) return fail(HELM_EINVAL, "ndim must be 2 or 3");
    if (n < 1 || ((n + 1) & n) != 0) return fail(HELM_EINVAL, "n must be 2^m - 1");
    if (n > (ndim == 2 ? 32767 : 2047)) return fail(HELM_EINVAL, "n beyond the library's grid bounds");
    if (!(h > 0.0)) return fail(HELM_EINVAL, "h must be positive");
    if (prec != HELM_PREC_FP64 && prec != HELM_PREC_MIXED) return fail(HELM_EINVAL, "bad precision");
    if (nu1 < 0 || nu1 > 8 || nu2 < 0 || nu2 > 8 || nu1 + nu2 < 1) return fail(HELM_EINVAL, "bad nu1/nu2");
    if (!device_ptr(rhs) || !device_ptr(e) || rhs == e) return fail(HELM_EINVAL, "bad rhs / e pointer");
    const int D = ndim;
    const int pr = (prec == HELM_PREC_FP64) ? 0 : 1;
    const size_t eb = pr == 0 ? 16 : 8;
    const int ttop = tail_top(D, pr == 0);
    const bool fused = (D == 2 && nu1 <= 4 && nu2 <= 4);

    InstDesc d;
    memset(&d, 0, sizeof d);
    d.D = D;
    d.n = n;
    d.h = h;
    int nl = 0, lt = -1;
    for (int m = n; m >= 1 && nl < HELM_MAXLEV; m = (m - 1) / 2) {
        if (lt < 0 && m <= ttop) lt = nl;
        d.lev[nl].n = m;
        ++nl;
    }
    if (lt < 0) return fail(HELM_EUNSUPPORTED, "hierarchy does not reach the tail size");
    d.nlev = nl;
    d.ltail = lt;
    size_t off = OFF_LEVELS;
    double hl = h;
    for (int l = 0; l < nl; ++l) {
        LevelDesc& L = d.lev[l];
        L.h = hl;
        hl *= 2.0;
        L.rows = L.n + 2;
        L.pitch = round_up(L.n + 2, 16);
        if (l > lt) continue;
        const size_t planes = (D == 3) ? (size_t)L.rows : 1;
        const size_t sz = a256((size_t)L.pitch * L.rows * planes * eb);
        const bool two = (D == 2 && l < lt);
        L.e = (void*)off;                      // offsets for now, pointers below
        L.rhs = (void*)(off + sz);
        if (two) L.e2 = (void*)(off + 2 * sz);
        off += (two ? 3 : 2) * sz;
    }
    set_shift(d, 0.0);                         // the alpha = k^2 cavity: Delta_h itself
    if (off > NOALLOC_BYTES) return fail(HELM_EUNSUPPORTED, "grid too large for the scratch array");
    unsigned char* base = nullptr;
    helm_status st = device_scratch(&base);
    if (st != HELM_OK) return st;
    for (int l = 0; l <= lt; ++l) {
        LevelDesc& L = d.lev[l];
        L.e = base + (size_t)L.e;
        L.rhs = base + (size_t)L.rhs;
        if (L.e2) L.e2 = base + (size_t)L.e2;
    }
    InstState s;
    memset(&s, 0, sizeof s);
    s.status = HELM_ST_ACTIVE;
    MgItem items[HELM_MAXLEV];
    for (int l = 0; l < HELM_MAXLEV; ++l) items[l] = MgItem{0, l};
    Header header;
    memset(&header, 0, sizeof header);
    memcpy(header.bytes, &d, sizeof d);
    memcpy(header.bytes + OFF_STATE, &s, sizeof s);
    memcpy(header.bytes + OFF_ITEMS, items, sizeof items);

    cudaStream_t sm = (cudaStream_t)cuda_stream;
    const InstDesc* dd = (const InstDesc*)base;
    const InstState* ds = (const InstState*)(base + OFF_STATE);
    const MgItem* di = (const MgItem*)(base + OFF_ITEMS);
#define NA_CK(call)                                                                     \
    do {                                                                                \
        if ((call) != cudaSuccess) return fail(HELM_ECUDA, #call);                      \
    } while (0)
    // rings of the level arrays must be zero; the previous call left its data here
    NA_CK(cudaMemsetAsync(base + OFF_LEVELS, 0, off - OFF_LEVELS, sm));
    k_noalloc_header<<<1, 256, 0, sm>>>(header, base);
    NA_CK(cudaGetLastError());
    NA_CK(launch_pack(D, pr, dd, 0, n, rhs, 1, sm));
    NA_CK(launch_pack(D, pr, dd, 0, n, e, 0, sm));
    auto pts = [&](int m) { return (D == 3) ? (long)m * m * m : (long)m * m; };
    if (fused) {
        for (int l = 0; l < lt; ++l)
            NA_CK(launch_down2d(pr, dd, ds, di + l, 1, tiles2d(d.lev[l].n), nu1, 1,
                                tile_shape2d(d.lev[l].n), sm));
        NA_CK(launch_tail(D, pr, d.lev[lt].n, dd, ds, di + lt, 1, nu1, nu2, 1, sm));
        for (int l = lt - 1; l >= 0; --l)
            NA_CK(launch_up2d(pr, dd, ds, di + l, 1, tiles2d(d.lev[l].n), nu2, tile_shape2d(d.lev[l].n),
                              nu1 == 0 ? 1 : 0, sm));
    } else {
        // without pre-smoothing the coarse iterates are zero on the way down: the
        // restriction takes rhs alone and the prolongation assigns (as poisson_vcycle)
        const int zmode = (nu1 == 0) ? 1 : 0;
        for (int l = 0; l < lt; ++l) {
            const int m = d.lev[l].n;
            const int w_rb = (int)(((D == 3) ? (long)m * m : m) * ((m + 1) / 2));
            for (int it = 0; it < nu1; ++it) {
                NA_CK(launch_rbgs(D, pr, dd, ds, di + l, 1, w_rb, 0, it == 0 ? 1 : 0, sm));
                NA_CK(launch_rbgs(D, pr, dd, ds, di + l, 1, w_rb, 1, 0, sm));
            }
            NA_CK(launch_restrict(D, pr, dd, ds, di + l, 1, (int)pts(d.lev[l + 1].n), sm, zmode));
        }
        NA_CK(launch_tail(D, pr, d.lev[lt].n, dd, ds, di + lt, 1, nu1, nu2, 1, sm));
        for (int l = lt - 1; l >= 0; --l) {
            const int m = d.lev[l].n;
            const int w_rb = (int)(((D == 3) ? (long)m * m : m) * ((m + 1) / 2));
            NA_CK(launch_prolong(D, pr, dd, ds, di + l, 1, (int)pts(m), sm, zmode, nu2 > 0 ? 1 : 0));
            for (int it = 0; it < nu2; ++it) {
                NA_CK(launch_rbgs(D, pr, dd, ds, di + l, 1, w_rb, 0, 0, sm));
                NA_CK(launch_rbgs(D, pr, dd, ds, di + l, 1, w_rb, 1, 0, sm));
            }
        }
    }
    NA_CK(launch_unpack(D, pr, dd, 0, n, e, sm));
#undef NA_CK
    return HELM_OK;
}
