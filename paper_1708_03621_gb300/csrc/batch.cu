// Batches of Hamiltonian applications replayed as one CUDA graph: many
// k-points of one cell (uneven sphere sizes) and independent cells with their
// own boxes run back to back from a single graph launch, with no host work
// between them.  (JDFTx distributes k-points over MPI processes, Sec. 3; on
// one GPU they become entries of one batch.)
//
// jdft_batch_create runs every item once on a private stream (growing each
// basis workspace to its final size, so no allocation happens afterwards),
// then captures the same calls into a graph and instantiates it.  The batch
// keeps the device pointers it was given; the caller keeps those buffers alive
// and fills the inputs before each jdft_batch_launch.
#include <vector>

#include "common.cuh"

struct jdft_batch_s {
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<jdft_apply_item> items;
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
        delete bt;
        return set_error(s, msg);
    };
    // the warm-up runs on a private stream and shares each basis workspace with
    // earlier calls on other streams: let all earlier device work finish first
    if (cudaDeviceSynchronize() != cudaSuccess)
        return fail(set_error(JDFT_ERR_CUDA, "jdft_batch_create: earlier device work failed"));
    if (cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(set_error(JDFT_ERR_CUDA, "jdft_batch_create: stream"));
    jdft_status s = run_items(bt->items, bt->stream);  // warm-up: workspaces reach their final size
    if (s != JDFT_OK) return fail(s);
    if (cudaStreamSynchronize(bt->stream) != cudaSuccess)
        return fail(set_error(JDFT_ERR_CUDA, "jdft_batch_create: warm-up failed"));
    jdft_profile_enable(0);
    if (cudaStreamBeginCapture(bt->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail(set_error(JDFT_ERR_CUDA, "jdft_batch_create: begin capture"));
    s = run_items(bt->items, bt->stream);
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
    delete bt;
    return JDFT_OK;
}

}  // extern "C"
