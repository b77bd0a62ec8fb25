// NCCL communication for slab-partitioned handles (st_comm_nccl_* in
// include/st_iga.h): the halo plane of the time coupling by ncclSend /
// ncclRecv, the gathered coarse level by ncclAllGather and the Krylov dot
// products by ncclAllReduce, all stream-ordered on the handle's stream.
//
// libnccl.so.2 is opened at run time (the process normally has it loaded
// already through PyTorch), so building the library needs no NCCL headers or
// link step.  Only the handful of entry points used here are declared, with
// the public NCCL signatures.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <cstring>
#include <mutex>

#include "../../include/st_iga.h"

namespace {

using ncclComm_t = void *;
struct ncclUniqueId {
    char internal[128];
};
using nccl_rc = int;            // ncclResult_t; 0 = success
constexpr int kUint8 = 1;       // ncclDataType_t values
constexpr int kFloat64 = 8;
constexpr int kSum = 0;         // ncclRedOp_t

struct Nccl {
    void *lib = nullptr;
    nccl_rc (*get_unique_id)(ncclUniqueId *) = nullptr;
    nccl_rc (*comm_init_rank)(ncclComm_t *, int, ncclUniqueId, int) = nullptr;
    nccl_rc (*comm_destroy)(ncclComm_t) = nullptr;
    nccl_rc (*group_start)() = nullptr;
    nccl_rc (*group_end)() = nullptr;
    nccl_rc (*send)(const void *, size_t, int, int, ncclComm_t, cudaStream_t) = nullptr;
    nccl_rc (*recv)(void *, size_t, int, int, ncclComm_t, cudaStream_t) = nullptr;
    nccl_rc (*all_gather)(const void *, void *, size_t, int, ncclComm_t, cudaStream_t) = nullptr;
    nccl_rc (*all_reduce)(const void *, void *, size_t, int, int, ncclComm_t, cudaStream_t) = nullptr;
};

std::mutex g_mu;
Nccl g_nccl;
bool g_tried = false;

template <typename F>
bool sym(void *lib, const char *name, F *out) {
    *out = reinterpret_cast<F>(dlsym(lib, name));
    return *out != nullptr;
}

const Nccl *nccl() {
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_tried) return g_nccl.lib ? &g_nccl : nullptr;
    g_tried = true;
    void *lib = dlopen("libnccl.so.2", RTLD_NOW | RTLD_GLOBAL);
    if (!lib) lib = dlopen("libnccl.so", RTLD_NOW | RTLD_GLOBAL);
    if (!lib) return nullptr;
    Nccl n;
    n.lib = lib;
    const bool ok = sym(lib, "ncclGetUniqueId", &n.get_unique_id) &&
                    sym(lib, "ncclCommInitRank", &n.comm_init_rank) &&
                    sym(lib, "ncclCommDestroy", &n.comm_destroy) &&
                    sym(lib, "ncclGroupStart", &n.group_start) &&
                    sym(lib, "ncclGroupEnd", &n.group_end) && sym(lib, "ncclSend", &n.send) &&
                    sym(lib, "ncclRecv", &n.recv) && sym(lib, "ncclAllGather", &n.all_gather) &&
                    sym(lib, "ncclAllReduce", &n.all_reduce);
    if (!ok) {
        dlclose(lib);
        return nullptr;
    }
    g_nccl = n;
    return &g_nccl;
}

struct Ctx {
    const Nccl *n = nullptr;
    ncclComm_t comm = nullptr;
    cudaStream_t stream = nullptr;  // for the host all-reduce
    double *buf = nullptr;          // device staging of the host all-reduce
    size_t cap = 0;
};

int cb_sendrecv(void *ctx, const void *send, int dst, void *recv, int src, size_t bytes,
                void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (c->n->group_start() != 0) return 1;
    if (dst >= 0 && c->n->send(send, bytes, kUint8, dst, c->comm, s) != 0) {
        c->n->group_end();
        return 1;
    }
    if (src >= 0 && c->n->recv(recv, bytes, kUint8, src, c->comm, s) != 0) {
        c->n->group_end();
        return 1;
    }
    return c->n->group_end() != 0;
}

int cb_allgather(void *ctx, const void *send, void *recv, size_t bytes, void *stream) {
    Ctx *c = static_cast<Ctx *>(ctx);
    return c->n->all_gather(send, recv, bytes, kUint8, c->comm,
                            static_cast<cudaStream_t>(stream)) != 0;
}

int cb_allreduce(void *ctx, double *vals, size_t count) {
    Ctx *c = static_cast<Ctx *>(ctx);
    if (count > c->cap) {
        if (c->buf) cudaFree(c->buf);
        c->buf = nullptr;
        c->cap = 0;
        if (cudaMalloc(&c->buf, count * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return 1;
        }
        c->cap = count;
    }
    if (cudaMemcpyAsync(c->buf, vals, count * sizeof(double), cudaMemcpyHostToDevice, c->stream) !=
        cudaSuccess)
        return 1;
    if (c->n->all_reduce(c->buf, c->buf, count, kFloat64, kSum, c->comm, c->stream) != 0) return 1;
    if (cudaMemcpyAsync(vals, c->buf, count * sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
        cudaSuccess)
        return 1;
    return cudaStreamSynchronize(c->stream) != cudaSuccess;
}

}  // namespace

extern "C" {

int st_comm_nccl_unique_id(void *unique_id) {
    if (!unique_id) return ST_ERR_INVALID_ARG;
    const Nccl *n = nccl();
    if (!n) return ST_ERR_UNSUPPORTED;
    ncclUniqueId id;
    if (n->get_unique_id(&id) != 0) return ST_ERR_COMM;
    std::memcpy(unique_id, &id, sizeof id);
    return ST_OK;
}

int st_comm_nccl_create(st_comm *out, int size, int rank, const void *unique_id) {
    if (!out || !unique_id || size < 1 || rank < 0 || rank >= size) return ST_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof *out);
    const Nccl *n = nccl();
    if (!n) return ST_ERR_UNSUPPORTED;
    Ctx *c = new Ctx();
    c->n = n;
    ncclUniqueId id;
    std::memcpy(&id, unique_id, sizeof id);
    if (n->comm_init_rank(&c->comm, size, id, rank) != 0) {
        delete c;
        return ST_ERR_COMM;
    }
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        n->comm_destroy(c->comm);
        delete c;
        return ST_ERR_CUDA;
    }
    out->rank = rank;
    out->size = size;
    out->host_buffers = 0;
    out->ctx = c;
    out->sendrecv = cb_sendrecv;
    out->allgather = cb_allgather;
    out->allreduce_sum = cb_allreduce;
    return ST_OK;
}

void st_comm_nccl_destroy(st_comm *cm) {
    if (!cm || !cm->ctx) return;
    Ctx *c = static_cast<Ctx *>(cm->ctx);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->buf) cudaFree(c->buf);
    if (c->comm) c->n->comm_destroy(c->comm);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
    cm->ctx = nullptr;
}

}  // extern "C"
