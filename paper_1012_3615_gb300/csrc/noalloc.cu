// bri_build_hops_noalloc: the hop precompute (path sums + SU(3) projection)
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: an application that routes every
// device allocation through its own pool and forbids others, or an embedding
// that must not grow its device footprint once it is running.  This entry
// point takes the links and an output buffer from the caller and keeps its
// only work space -- the path sums of all 81 offsets -- in a file-scope device
// array of fixed size, so it allocates nothing.
//
// Limits and sharing rules:
//  - at most BRI_NOALLOC_MAX_SITES sites (81 x 144 bytes of scratch per site,
//    about 45.6 MiB that every GPU loading the library holds until exit);
//  - every call uses the same array, so calls that overlap on the GPU (two
//    streams, two host threads) race and must be serialised by the caller;
//  - nothing has to start at zero: each call writes every scratch entry it
//    reads before reading it (level n is written before level n+1 reads it).
//  - the first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current; make that first call
//    before any stream capture.  The address is cached per device together
//    with the identity of the device's current context, and looked up again
//    when the context changes (a cudaDeviceReset destroys the primary context
//    and the module holding the array is loaded anew, possibly elsewhere).
#include <cudaTypedefs.h>

#include <cstring>
#include <string>

#include "ctx.h"
#include "project.cuh"

using namespace bri;

#define BRI_NOALLOC_MAX_SITES 4096
#define BRI_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char
    g_hop_scratch[(size_t)NOFF * BRI_NOALLOC_MAX_SITES * sizeof(M3<double2>)];

namespace {

void *g_scratch_addr[BRI_NOALLOC_MAX_DEVICES];
bool g_scratch_ready[BRI_NOALLOC_MAX_DEVICES];
unsigned long long g_scratch_ctx[BRI_NOALLOC_MAX_DEVICES];  // context id the address belongs to

// unique id of the context current on this thread (0 if it cannot be read);
// the driver calls are reached through the runtime, so the library does not
// link against the driver library itself
unsigned long long current_context_id() {
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess)
            get_current = (PFN_cuCtxGetCurrent_v4000)f1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess)
            get_id = (PFN_cuCtxGetId_v12000)f2;
        looked_up = true;
    }
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// offsets of hop class n, packed class after class
struct ClassList {
    int k[NOFF];
    int start[6];
};

// one level of the averaging recursion over the first step of every path
__global__ void k_na_level(int n, ClassList cl, const double2 *__restrict__ U, M3<double2> *__restrict__ A, Geom g) {
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    const int idx = cl.start[n] + blockIdx.y;
    if (site >= g.V || idx >= cl.start[n + 1]) return;
    const int k = cl.k[idx];
    int x[4];
    SiteNb nb = site_nb(g, site, x);
    M3<double2> acc = m3_zero<double2>();
    int p3 = 1;
    for (int mu = 0; mu < 4; mu++, p3 *= 3) {
        const int c = (k / p3) % 3 - 1;
        if (c == 0) continue;
        M3<double2> F;
        const double2 *u = U + ((size_t)(c > 0 ? site : site + nb.bw[mu]) * 4 + mu) * 9;
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) F.e[3 * i + j] = c > 0 ? u[3 * i + j] : cconj(u[3 * j + i]);
        if (n == 1) {
            acc = F;
        } else {
            const int y = site + (c > 0 ? nb.fw[mu] : nb.bw[mu]);
            acc = m3_mad(acc, F, A[(size_t)(k - c * p3) * g.V + y]);
        }
    }
    for (int i = 0; i < 9; i++) acc.e[i] = cscale(acc.e[i], 1.0 / n);
    A[(size_t)k * g.V + site] = acc;
}

// canonical field j (offset index j + 41) of every site, projected, into W [V][40][9]
__global__ void k_na_project(const M3<double2> *__restrict__ A, double2 *__restrict__ W, Geom g) {
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (site >= g.V) return;
    const int k = canon_k(j);
    const M3<double2> a = A[(size_t)k * g.V + site];
    const M3<double2> w = off_class(k) == 1 ? a : project_su3(a);
    for (int e = 0; e < 9; e++) W[((size_t)site * NCANON + j) * 9 + e] = w.e[e];
}

// errors of this stateless entry point are reported through bri_last_error(NULL)
bri_status fail(bri_status st, const std::string &msg) { return bri_fail(nullptr, st, msg); }

}  // namespace

extern "C" bri_status bri_build_hops_noalloc(const bri_lattice *lat, const double *U, double *W, void *stream) {
    if (!lat || !U || !W) return fail(BRI_EINVAL, "bri_build_hops_noalloc: null argument");
    if (((uintptr_t)U & 15u) || ((uintptr_t)W & 15u))
        return fail(BRI_EINVAL, "bri_build_hops_noalloc: U and W must be 16-byte aligned device pointers");
    Geom g;
    long long V = 1;
    for (int mu = 0; mu < 4; mu++) {
        if (lat->L[mu] < 3) return fail(BRI_EINVAL, "bri_build_hops_noalloc: lattice extents must be >= 3");
        if (lat->bc_sign[mu] != 1 && lat->bc_sign[mu] != -1)
            return fail(BRI_EINVAL, "bri_build_hops_noalloc: bc_sign must be +1 or -1");
        g.L[mu] = lat->L[mu];
        g.bc[mu] = lat->bc_sign[mu];
        V *= lat->L[mu];
    }
    if (V > BRI_NOALLOC_MAX_SITES)
        return fail(BRI_EINVAL, "bri_build_hops_noalloc: lattice volume exceeds the 4096-site scratch");
    g.V = (int)V;
    g.s0 = 0;
    g.s1 = (int)V;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= BRI_NOALLOC_MAX_DEVICES)
        return fail(BRI_ECUDA, "bri_build_hops_noalloc: no usable current device");
    // make the device's primary context current (initialising it if needed)
    // so that its identity can be compared with the cached one
    if (cudaSetDevice(dev) != cudaSuccess) return fail(BRI_ECUDA, "bri_build_hops_noalloc: cudaSetDevice failed");
    const unsigned long long ctx_id = current_context_id();
    if (!g_scratch_ready[dev] || ctx_id == 0 || ctx_id != g_scratch_ctx[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_hop_scratch);
        if (e != cudaSuccess || !p)
            return fail(BRI_ECUDA, std::string("bri_build_hops_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = ctx_id;
        g_scratch_ready[dev] = true;
    }
    M3<double2> *A = (M3<double2> *)g_scratch_addr[dev];
    ClassList cl;
    int cnt = 0;
    cl.start[0] = 0;
    for (int n = 1; n <= 4; n++) {
        cl.start[n] = cnt;
        for (int k = 0; k < NOFF; k++)
            if (off_class(k) == n) cl.k[cnt++] = k;
    }
    cl.start[5] = cnt;
    cudaStream_t s = (cudaStream_t)stream;
    const int T = 128;
    const unsigned nbx = (unsigned)((g.V + T - 1) / T);
    for (int n = 1; n <= 4; n++) {
        k_na_level<<<dim3(nbx, (unsigned)(cl.start[n + 1] - cl.start[n])), T, 0, s>>>(n, cl, (const double2 *)U, A, g);
        if (cudaGetLastError() != cudaSuccess) return fail(BRI_ECUDA, "bri_build_hops_noalloc: launch failed");
    }
    k_na_project<<<dim3(nbx, NCANON), T, 0, s>>>(A, (double2 *)W, g);
    if (cudaGetLastError() != cudaSuccess) return fail(BRI_ECUDA, "bri_build_hops_noalloc: launch failed");
    return BRI_OK;
}
