// jdft_apply_H_noalloc: the Hamiltonian application with no device allocation.
//
// jdft_apply_H keeps its intermediate column buffer in a basis-owned workspace
// that grows with cudaMalloc on first use.  Some callers cannot allow that:
// callers with a fixed memory budget or their own pool allocator that must see
// every device byte the process uses, and real-time loops where a
// synchronising allocation is not acceptable.  This
// entry point instead uses one fixed scratch array compiled into the library
// as a file-scope __device__ variable: every GPU that loads the library holds
// it (kNoAllocScratchBytes) until the process exits, and the call itself
// allocates nothing.
//
// Host code may not pass the array's name to a kernel (in host code the name
// denotes a host-side shadow, not device memory), so on the first call on
// each device the library asks the runtime for the device address with
// cudaGetSymbolAddress and caches it.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "chain.cuh"
#include "gemm.cuh"

namespace jdft {

constexpr size_t kNoAllocScratchBytes = 32u << 20;  // 32 MiB per device
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on first use).
static jdft_status noalloc_scratch(void** out) {
    int dev = 0;
    JDFT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return set_error(JDFT_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return set_error(JDFT_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return JDFT_OK;
}

static size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// Scratch bytes for a chunk of n bands: column buffer, then the nonlocal term's
// FP64 P^dag C block and its product-type D (P^dag C) block.
template <typename T>
static size_t chunk_bytes(const ChainGeom& g, int nproj, int n) {
    size_t b = round256((size_t)n * g.S2 * g.ncols * sizeof(c_t<T>));
    if (nproj > 0) b += round256((size_t)nproj * n * sizeof(double2)) + round256((size_t)nproj * n * sizeof(c_t<T>));
    return b;
}

template <typename T>
static jdft_status apply_noalloc(jdft_basis_s* b, int ik, const void* C, int ldc, void* HC, int ldhc, int nb,
                                 jdft_prec prec, cudaStream_t st) {
    const ChainGeom g = make_geom(b, ik);
    const KSphere& sp = b->ks[ik];
    if (chunk_bytes<T>(g, sp.nproj, 1) > kNoAllocScratchBytes)
        return set_error(JDFT_ERR_ARG, "jdft_apply_H_noalloc: one band needs more than the 32 MiB static scratch; "
                                       "use jdft_apply_H");
    int nc = 1;
    while (nc < nb && chunk_bytes<T>(g, sp.nproj, nc + 1) <= kNoAllocScratchBytes) ++nc;
    void* scratch = nullptr;
    jdft_status s = noalloc_scratch(&scratch);
    if (s != JDFT_OK) return s;
    const c_t<T>* tw = std::is_same<T, double>::value ? (const c_t<T>*)b->tw64 : (const c_t<T>*)b->tw32;
    const T* Vp = std::is_same<T, double>::value ? (const T*)b->V : (const T*)b->V32;
    const T* kin = std::is_same<T, double>::value ? (const T*)sp.kin : (const T*)sp.kin32;
    c_t<T>* colbuf = (c_t<T>*)scratch;
    const T omega = (T)b->omega, invN = (T)(1.0 / (double)b->N);
    for (int b0 = 0; b0 < nb; b0 += nc) {
        const int n = std::min(nc, nb - b0);
        const c_t<T>* Cc = (const c_t<T>*)C + (size_t)b0 * ldc;
        c_t<T>* Hc = (c_t<T>*)HC + (size_t)b0 * ldhc;
        if ((s = launch_zpass_inverse<T>(g, Cc, ldc, colbuf, n, tw, st))) return s;
        if ((s = launch_plane_apply<T>(g, colbuf, Vp, n, tw, st))) return s;
        if ((s = launch_zpass_forward<T, 0>(g, colbuf, Cc, ldc, Hc, ldhc, n, kin, omega, invN, tw, st))) return s;
        if (sp.nproj > 0) {
            void* nl = (char*)scratch + round256((size_t)n * g.S2 * g.ncols * sizeof(c_t<T>));
            if ((s = nonlocal_accumulate<T>(sp, Cc, ldc, Hc, ldhc, n, prec, nl, st))) return s;
        }
    }
    return JDFT_OK;
}

}  // namespace jdft

using namespace jdft;

extern "C" jdft_status jdft_apply_H_noalloc(jdft_basis_t b, int ik, const void* C, int ldc, void* HC, int ldhc, int nb,
                                            jdft_prec prec, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(b, "null basis");
    JDFT_CHECK_ARG(ik >= 0 && ik < b->nk, "k-point index out of range");
    JDFT_CHECK_ARG(nb >= 0, "nb must be >= 0");
    JDFT_CHECK_ARG(prec == JDFT_FP64 || prec == JDFT_FP32 || prec == JDFT_TF32X3 || prec == JDFT_BF16X3,
                   "unknown precision");
    if (nb == 0) return JDFT_OK;
    const int npw = b->ks[ik].npw;
    const uintptr_t align = prec == JDFT_FP64 ? 16 : 8;
    JDFT_CHECK_ARG(C && HC, "C or HC is null");
    JDFT_CHECK_ARG(ldc >= npw && ldhc >= npw, "leading dimension < npw");
    JDFT_CHECK_ARG((uintptr_t)C % align == 0 && (uintptr_t)HC % align == 0, "C or HC not aligned to its complex type");
    if (!b->have_V) return set_error(JDFT_ERR_ARG, "no potential set (call jdft_set_potential first)");
    cudaStream_t st = (cudaStream_t)stream;
    return prec == JDFT_FP64 ? apply_noalloc<double>(b, ik, C, ldc, HC, ldhc, nb, prec, st)
                             : apply_noalloc<float>(b, ik, C, ldc, HC, ldhc, nb, prec, st);
}
