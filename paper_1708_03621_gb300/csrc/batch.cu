// Batches of Hamiltonian applications replayed as one CUDA graph: many
// k-points of one cell (uneven sphere sizes) and independent cells with their
// own boxes run back to back from a single graph launch, with no host work
// between them.  (JDFTx distributes k-points over MPI processes, Sec. 3; on
// one GPU they become entries of one batch.)
//
// jdft_batch_create runs every item once on a private stream (growing each
// basis workspace to its final size, so no allocation happens afterwards),
// then captures the same calls into a graph and instantiates it.  When all
// items are k-points of one basis on a box the band-pair kernels serve, the
// FFT chain runs k-batched instead: one launch per stage (z pass in, plane
// pass, z pass out) over all items, each with its own sphere maps and column
// buffer (owned by the batch), then each item's projector term.  The batch
// keeps the device pointers it was given; the caller keeps those buffers alive
// and fills the inputs before each jdft_batch_launch.
#include <algorithm>
#include <vector>

#include "chain.cuh"
#include "common.cuh"
#include "gemm.cuh"

struct jdft_batch_s {
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<jdft_apply_item> items;
    // k-batched chain (items of one basis on a box with band-pair kernels):
    // one launch per FFT stage over all items, then each item's projector term
    bool kbatch = false;
    void* kmem = nullptr;  // column buffers, job table, projector-term scratch
    std::vector<jdft::ChainGeom> gs;
    jdft::KJob* djobs = nullptr;
    void* nlwork = nullptr;
    int64_t items_total = 0;
    int max_ncols = 0, max_nb = 0;
};

using namespace jdft;

extern "C" jdft_status jdft_profile_enable(int on);

static jdft_status run_items(const std::vector<jdft_apply_item>& items, cudaStream_t st) {
    for (const auto& it : items) {
        jdft_status s = jdft_apply_H(it.basis, it.ik, it.C, it.ldc, it.HC, it.ldhc, it.nb, it.prec, st);
        if (s != JDFT_OK) return s;
    }
    return JDFT_OK;
}

static size_t r256(size_t x) { return (x + 255) / 256 * 256; }

// Whether the items can run as one k-batched chain: two or more items, one
// basis with a potential, FP32 blocks, well-formed blocks, and a box the
// band-pair plane kernels and the register z passes are compiled for.
static bool kbatch_eligible(const std::vector<jdft_apply_item>& items) {
    if (items.size() < 2) return false;
    jdft_basis_s* b = items[0].basis;
    if (!b || !b->have_V) return false;
    const int fast_z[] = {12, 16, 40, 48, 64, 80, 128, 256};
    if (std::find(std::begin(fast_z), std::end(fast_z), b->S[2]) == std::end(fast_z)) return false;
    if (!plane_pair_batch_supported(make_geom(b, 0))) return false;
    for (const auto& it : items) {
        if (it.basis != b || it.prec != items[0].prec || it.prec == JDFT_FP64) return false;
        if (it.ik < 0 || it.ik >= b->nk || it.nb < 1 || !it.C || !it.HC) return false;
        const int npw = b->ks[it.ik].npw;
        if (it.ldc < npw || it.ldhc < npw || (uintptr_t)it.C % 8 || (uintptr_t)it.HC % 8) return false;
    }
    return true;
}

// Column buffers, the device job table and the projector-term scratch of a
// k-batched batch.
static jdft_status kbatch_setup(jdft_batch_s* bt) {
    jdft_basis_s* b = bt->items[0].basis;
    size_t off = 0, nl = 0;
    std::vector<size_t> col_off;
    for (const auto& it : bt->items) {
        const ChainGeom g = make_geom(b, it.ik);
        col_off.push_back(off);
        off += r256((size_t)it.nb * g.S2 * g.ncols * sizeof(float2));
        const KSphere& sp = b->ks[it.ik];
        nl = std::max(nl, nonlocal_workspace_bytes(sp.nproj, it.nb, sizeof(float2), sp.npw, it.prec, true, true));
    }
    const size_t jobs_off = off;
    off += r256(bt->items.size() * sizeof(KJob));
    const size_t nl_off = off;
    off += r256(nl);
    JDFT_CUDA_TRY(cudaMalloc(&bt->kmem, std::max<size_t>(off, 256)));
    char* base = (char*)bt->kmem;
    std::vector<KJob> jobs;
    int64_t item0 = 0;
    for (size_t i = 0; i < bt->items.size(); ++i) {
        const auto& it = bt->items[i];
        KJob j;
        j.g = make_geom(b, it.ik);
        j.C = (const float2*)it.C;
        j.ldc = it.ldc;
        j.HC = (float2*)it.HC;
        j.ldhc = it.ldhc;
        j.colbuf = (float2*)(base + col_off[i]);
        j.kin = b->ks[it.ik].kin32;
        j.nb = it.nb;
        j.item0 = item0;
        item0 += (int64_t)j.g.S2 * ((it.nb + 1) / 2);
        bt->max_ncols = std::max(bt->max_ncols, j.g.ncols);
        bt->max_nb = std::max(bt->max_nb, it.nb);
        bt->gs.push_back(j.g);
        jobs.push_back(j);
    }
    bt->items_total = item0;
    bt->djobs = (KJob*)(base + jobs_off);
    bt->nlwork = base + nl_off;
    JDFT_CUDA_TRY(cudaMemcpy(bt->djobs, jobs.data(), jobs.size() * sizeof(KJob), cudaMemcpyHostToDevice));
    return JDFT_OK;
}

// The k-batched chain: z pass in, plane pass and z pass out over all items in
// one launch each, then every item's projector term.
static jdft_status run_kbatch(jdft_batch_s* bt, cudaStream_t st) {
    jdft_basis_s* b = bt->items[0].basis;
    const ChainGeom& g = bt->gs[0];
    const int nj = (int)bt->items.size();
    const float2* tw2 = b->tw32 + g.p2.tw_offset;
    jdft_status s;
    if ((s = launch_zpass_inverse_batch(g, bt->djobs, nj, bt->max_ncols, bt->max_nb, tw2, st))) return s;
    if ((s = launch_plane_apply_pair_batch(bt->gs, bt->djobs, bt->items_total, b->V32, b->tw32, st))) return s;
    if ((s = launch_zpass_forward_batch(g, bt->djobs, nj, bt->max_ncols, bt->max_nb, (float)b->omega,
                                        (float)(1.0 / (double)b->N), tw2, st)))
        return s;
    for (const auto& it : bt->items) {
        const KSphere& sp = b->ks[it.ik];
        if ((s = nonlocal_accumulate<float>(sp, it.C, it.ldc, it.HC, it.ldhc, it.nb, it.prec, bt->nlwork, st, true,
                                            nullptr, true)))
            return s;
    }
    return JDFT_OK;
}

static jdft_status run_batch(jdft_batch_s* bt, cudaStream_t st) {
    return bt->kbatch ? run_kbatch(bt, st) : run_items(bt->items, st);
}

extern "C" {

jdft_status jdft_batch_create(int n, const jdft_apply_item* items, jdft_batch_t* out) {
    clear_error();
    JDFT_CHECK_ARG(n >= 1 && items && out, "bad arguments");
    *out = nullptr;
    jdft_batch_s* bt = new jdft_batch_s();
    bt->items.assign(items, items + n);
    auto fail = [&](jdft_status s) {
        std::string msg = jdft_last_error();
        if (bt->exec) cudaGraphExecDestroy(bt->exec);
        if (bt->graph) cudaGraphDestroy(bt->graph);
        if (bt->stream) cudaStreamDestroy(bt->stream);
        if (bt->kmem) cudaFree(bt->kmem);
        delete bt;
        return set_error(s, msg);
    };
    // the warm-up runs on a private stream and shares each basis workspace with
    // earlier calls on other streams: let all earlier device work finish first
    if (cudaDeviceSynchronize() != cudaSuccess)
        return fail(set_error(JDFT_ERR_CUDA, "jdft_batch_create: earlier device work failed"));
    if (cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(set_error(JDFT_ERR_CUDA, "jdft_batch_create: stream"));
    jdft_status s = JDFT_OK;
    if (kbatch_eligible(bt->items)) {
        bt->kbatch = true;
        if ((s = kbatch_setup(bt)) != JDFT_OK) return fail(s);
    }
    s = run_batch(bt, bt->stream);  // warm-up: workspaces reach their final size
    if (s != JDFT_OK) return fail(s);
    if (cudaStreamSynchronize(bt->stream) != cudaSuccess)
        return fail(set_error(JDFT_ERR_CUDA, "jdft_batch_create: warm-up failed"));
    jdft_profile_enable(0);
    if (cudaStreamBeginCapture(bt->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail(set_error(JDFT_ERR_CUDA, "jdft_batch_create: begin capture"));
    s = run_batch(bt, bt->stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(bt->stream, &g);
    if (s != JDFT_OK) {
        if (g) cudaGraphDestroy(g);
        return fail(s);
    }
    if (e != cudaSuccess || !g)
        return fail(set_error(JDFT_ERR_CUDA, std::string("jdft_batch_create: capture: ") + cudaGetErrorString(e)));
    bt->graph = g;
    e = cudaGraphInstantiate(&bt->exec, g, 0);
    if (e != cudaSuccess)
        return fail(set_error(JDFT_ERR_CUDA, std::string("jdft_batch_create: instantiate: ") + cudaGetErrorString(e)));
    *out = bt;
    return JDFT_OK;
}

jdft_status jdft_batch_launch(jdft_batch_t bt, void* stream) {
    clear_error();
    JDFT_CHECK_ARG(bt, "null batch");
    JDFT_CUDA_TRY(cudaGraphLaunch(bt->exec, (cudaStream_t)stream));
    return JDFT_OK;
}

jdft_status jdft_batch_destroy(jdft_batch_t bt) {
    if (!bt) return JDFT_OK;
    if (bt->stream) cudaStreamSynchronize(bt->stream);
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->graph) cudaGraphDestroy(bt->graph);
    if (bt->stream) cudaStreamDestroy(bt->stream);
    if (bt->kmem) cudaFree(bt->kmem);
    delete bt;
    return JDFT_OK;
}

int jdft_batch_is_kbatched(jdft_batch_t bt) { return bt && bt->kbatch ? 1 : 0; }

}  // extern "C"
