// p2s_fill_elements_noalloc: the fill of p2s_fill_elements without any device allocation.
//
// Who needs it: programs that must not call cudaMalloc/cudaFree while they run, for
// example a solver that hands all free device memory to its own pool at start-up and
// never returns any, a service that runs under a fixed device-memory budget, or a loop
// that cannot afford the device-wide synchronisation a cudaMalloc/cudaFree may cause.
// Such a caller creates a context once (p2s_create, which does allocate its small
// read-only tables) and afterwards fills elements through this entry point only.
//
// Where the scratch lives: one file-scope array in device memory (g_noalloc_scratch,
// 18.3 MiB), present on every GPU that loads this library until the process exits.
// It holds the moment tensors between the two kernels, the per-element descriptors,
// the contraction work list and the two work-queue counters (contraction units, moment
// elements).  Its device address is taken once per device with cudaGetSymbolAddress, by
// p2s_create (noalloc_prepare below), with that device current: the host-side name of
// the array is only a stand-in and must never be passed to a kernel.  Doing the look-up
// there matters because the runtime may load this file's module (and place the array in
// device memory) only when the address is first asked for; a caller that has handed all
// free device memory to its own pool after p2s_create must not meet that load inside
// the fill.
#include <cstring>
#include <mutex>

#include "p2s_internal.h"

namespace p2s {
namespace {

constexpr int64_t kNaMaxElems = 2048;
constexpr int64_t kNaMaxMoments = int64_t(1) << 21;  // 8-byte moment entries (16 MiB)
constexpr int64_t kNaMaxUnits = int64_t(1) << 17;    // contraction work units

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kNaMomBytes = align256(sizeof(double) * kNaMaxMoments);
constexpr size_t kNaDescBytes = align256(sizeof(ElemDesc) * kNaMaxElems);
constexpr size_t kNaUnitBytes = align256(sizeof(ContractUnit) * kNaMaxUnits);
constexpr size_t kNaCounterBytes = 256;
constexpr size_t kNaBytes = kNaMomBytes + kNaDescBytes + kNaUnitBytes + kNaCounterBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;                   // serialises the host staging below
unsigned char* g_na_addr[kNaMaxDevices];  // device address of the scratch, per device
ElemDesc g_na_desc[kNaMaxElems];         // host staging of the descriptors
ContractUnit g_na_units[kNaMaxUnits];    // host staging of the work list

}  // namespace

// Called by p2s_create with `device` current: look the array up once for this device.
int noalloc_prepare(int device) {
    if (device < 0 || device >= kNaMaxDevices) return P2S_OK;  // the fill refuses such devices
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (g_na_addr[device]) return P2S_OK;
    void* ptr = nullptr;
    const cudaError_t ce = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (ce != cudaSuccess) return fail(P2S_ERR_CUDA, "p2s_create: cudaGetSymbolAddress of the no-alloc scratch", ce);
    g_na_addr[device] = static_cast<unsigned char*>(ptr);
    return P2S_OK;
}

}  // namespace p2s

using namespace p2s;

extern "C" int p2s_fill_elements_noalloc(p2s_ctx* ctx, const p2s_geometry* geom, const p2s_material* mat,
                                         const p2s_orders* orders, const p2s_quadrature* quad,
                                         const p2s_fill_opts* opts, double* out, int32_t* elem_status,
                                         void* stream) {
    const DeviceTables* T = context_tables(ctx);
    if (!T || !geom) return fail(P2S_ERR_ARG, "p2s_fill_elements_noalloc: NULL context or geometry");
    const int64_t E = geom->n_elem;
    if (E < 0) return fail(P2S_ERR_ARG, "p2s_fill_elements_noalloc: negative n_elem");
    if (E > kNaMaxElems)
        return fail(P2S_ERR_BUFFER, "p2s_fill_elements_noalloc: more than 2048 elements in one call");
    if (T->device < 0 || T->device >= kNaMaxDevices)
        return fail(P2S_ERR_ARG, "p2s_fill_elements_noalloc: device index above 63");

    std::lock_guard<std::mutex> lock(g_na_mutex);
    cudaError_t ce = cudaSetDevice(T->device);
    if (ce != cudaSuccess) return fail(P2S_ERR_CUDA, "p2s_fill_elements_noalloc: cudaSetDevice", ce);
    unsigned char* base = g_na_addr[T->device];  // looked up by p2s_create
    if (!base) return fail(P2S_ERR_CUDA, "p2s_fill_elements_noalloc: scratch address missing for this device");
    void* d_mom = base;
    ElemDesc* d_desc = reinterpret_cast<ElemDesc*>(base + kNaMomBytes);
    ContractUnit* d_units = reinterpret_cast<ContractUnit*>(base + kNaMomBytes + kNaDescBytes);
    unsigned long long* d_counter =
        reinterpret_cast<unsigned long long*>(base + kNaMomBytes + kNaDescBytes + kNaUnitBytes);

    UnitSink sink;
    sink.buf = g_na_units;
    sink.cap = kNaMaxUnits;
    PlanLayout L;
    int rc = build_layout(*T, E, orders, quad, opts, g_na_desc, sink, L);
    if (rc) return rc;
    if (sink.overflow())
        return fail(P2S_ERR_BUFFER, "p2s_fill_elements_noalloc: work list above 131072 units; fill fewer elements");
    if (L.mom_entries > kNaMaxMoments)
        return fail(P2S_ERR_BUFFER, "p2s_fill_elements_noalloc: moments above 2097152 entries; fill fewer elements");
    if (E == 0) return P2S_OK;
    if (!out) return fail(P2S_ERR_ARG, "p2s_fill_elements_noalloc: NULL out");

    cudaStream_t s = (cudaStream_t)stream;
    // The staging arrays are pageable host memory: each copy has left them before it
    // returns, so the next call may refill them.
    ce = cudaMemcpyAsync(d_desc, g_na_desc, sizeof(ElemDesc) * E, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess && L.n_units)
        ce = cudaMemcpyAsync(d_units, g_na_units, sizeof(ContractUnit) * L.n_units, cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) return fail(P2S_ERR_CUDA, "p2s_fill_elements_noalloc: upload", ce);
    rc = run_moments(*T, L, d_desc, geom, mat, d_mom, elem_status, s, d_counter + 1);
    if (rc) return rc;
    // run_contract clears the queue counter on the stream before its launch
    return run_contract(*T, L, d_desc, d_units, d_counter, d_mom, out, s);
}
