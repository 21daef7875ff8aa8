// Allocation-free variant of the GPU direct sum (fmm_layered_direct_noalloc).
//
// Some callers cannot allocate device memory at the point where they need the
// potentials: code that runs inside another framework's memory manager (whose
// caching allocator already owns the free device memory), or an inner solver
// loop that must not call cudaMalloc/cudaFree because those calls synchronize
// the whole device.  This entry point does the same work as
// fmm_layered_direct but keeps its scratch (the per-node reaction
// coefficients, the interface-distance reductions and the error flags) in one
// file-scope device array of fixed size instead of the handle's growable
// workspace.  It only reads what fmm_layered_create built (the quadrature rule
// and the reaction densities) and allocates nothing.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "fmm_internal.h"

// Fixed scratch; every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FMM_NOALLOC_SCRATCH_BYTES];

// Host code cannot use g_noalloc_scratch's name as a device address: the
// address is fetched once per device with cudaGetSymbolAddress.
static std::mutex g_scratch_mu;
static void* g_scratch_ptr[64] = {nullptr};

static void* scratch_address(int dev) {
  if (dev < 0 || dev >= 64) throw FmmError(FMM_ERR_UNSUPPORTED, "device index out of range for the fixed scratch");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      throw FmmError(FMM_ERR_CUDA, std::string("cudaGetSymbolAddress of the fixed scratch failed: ") +
                                       cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

void launch_coef(int L1, const Rule& R, cplx* coef, cudaStream_t st);
RuleView make_rule_view(const Rule& R, const cplx* coef);
SurrView surrogate_view(const fmm_layered* h);
void launch_direct(long nt, const double* tgt, long ns, const double* src, const double* q, DirectMedium md,
                   RuleView R, const cplx* coef_all, double* out, cudaStream_t st);
void launch_norm_paper(long n, const double* tgt, DirectMedium md, double* out, cudaStream_t st);

__device__ inline unsigned long long na_enc(double x) {
  unsigned long long u = __double_as_longlong(x);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ULL);
}

// Per point: finiteness, on-interface check and the smallest distance of the
// point to an interface of its layer (min over sources in red[0], targets in red[1]).
__global__ void k_noalloc_scan(long n, const double* __restrict__ xyz, const double* __restrict__ q, int set,
                               DirectMedium md, unsigned long long* __restrict__ red, int* __restrict__ flags) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
  bool fin = isfinite(x) && isfinite(y) && isfinite(z);
  if (q) fin = fin && isfinite(q[2 * i]) && isfinite(q[2 * i + 1]);
  if (!fin) {
    atomicOr(flags, 2);
    return;
  }
  const PointLayer pl = classify_height(z, md.d, md.L1);
  if (pl.on_iface) atomicOr(flags, 1);
  const double g = fmin(pl.gap_below, pl.gap_above);
  if (isfinite(g)) atomicMin(&red[set], na_enc(g));
}

extern "C" int fmm_layered_direct_noalloc(fmm_layered_t* h, long ns, const double* src, const double* q, long nt,
                                          const double* tgt, double* out, void* stream) {
  if (!h) return FMM_ERR_ARG;
  h->err.clear();
  if (ns < 0 || nt < 0 || (ns && (!src || !q)) || (nt && (!tgt || !out))) {
    h->err = "invalid argument";
    return FMM_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  try {
    const Rule& R = h->rule;
    const int Q = R.Q();
    const size_t coef_bytes = sizeof(cplx) * (size_t)h->L1 * h->L1 * 4 * Q;
    const size_t head = 256;      // reductions and flags, then the coefficient table
    if (head + coef_bytes > (size_t)FMM_NOALLOC_SCRATCH_BYTES)
      throw FmmError(FMM_ERR_UNSUPPORTED,
                     "the reaction coefficient table (" + std::to_string(coef_bytes) + " bytes for " +
                         std::to_string(h->L1) + " layers and " + std::to_string(Q) +
                         " quadrature nodes) exceeds the fixed scratch of " +
                         std::to_string((long)FMM_NOALLOC_SCRATCH_BYTES) + " bytes");
    if (nt == 0) return FMM_OK;
    int dev = 0;
    FMM_CHECK(cudaGetDevice(&dev));
    unsigned char* base = (unsigned char*)scratch_address(dev);
    unsigned long long* red = (unsigned long long*)base;      // [2]
    int* flags = (int*)(base + 16);
    cplx* coef = (cplx*)(base + head);
    DirectMedium md{};
    md.L1 = h->L1;
    for (int l = 0; l < h->L1; ++l) md.k[l] = h->k[l];
    for (size_t j = 0; j < h->d.size(); ++j) md.d[j] = h->d[j];
    // the scratch keeps the previous call's contents: reset what must start cleared
    FMM_CHECK(cudaMemsetAsync(red, 0xFF, 16, st));
    FMM_CHECK(cudaMemsetAsync(flags, 0, 4, st));
    if (ns) LAUNCH(k_noalloc_scan<<<(ns + 255) / 256, 256, 0, st>>>(ns, src, q, 0, md, red, flags));
    LAUNCH(k_noalloc_scan<<<(nt + 255) / 256, 256, 0, st>>>(nt, tgt, nullptr, 1, md, red, flags));
    FMM_CHECK(cudaGetLastError());
    unsigned long long hred[2];
    int hflags = 0;
    FMM_CHECK(cudaMemcpyAsync(hred, red, 16, cudaMemcpyDeviceToHost, st));
    FMM_CHECK(cudaMemcpyAsync(&hflags, flags, 4, cudaMemcpyDeviceToHost, st));
    FMM_CHECK(cudaStreamSynchronize(st));
    if (hflags & 2) throw FmmError(FMM_ERR_NONFINITE, "non-finite coordinate or charge");
    if (hflags & 1) throw FmmError(FMM_ERR_ON_INTERFACE, "a point lies exactly on an interface");
    if (h->L1 > 1 && ns > 0) {
      auto dec = [](unsigned long long e) {
        unsigned long long u = (e >> 63) ? (e & 0x7FFFFFFFFFFFFFFFULL) : ~e;
        double x;
        memcpy(&x, &u, 8);
        return x;
      };
      double gsum = dec(hred[0]) + dec(hred[1]);
      if (!R.covers(R.near_tmax(gsum)))
        throw FmmError(FMM_ERR_UNSUPPORTED,
                       "the quadrature rule held by the handle is too short for these points and growing it "
                       "would allocate: run fmm_layered_direct or fmm_layered_eval once on this geometry first");
    }
    launch_coef(h->L1, R, coef, st);
    // the trained surrogate (FMM_SURROGATE) is read from the handle as in
    // fmm_layered_direct: its weights and cell verdicts already exist
    RuleView rv = make_rule_view(R, coef);
    rv.surr = surrogate_view(h);
    launch_direct(nt, tgt, ns, src, q, md, rv, coef, out, st);
    if (h->flags & FMM_NORM_PAPER) launch_norm_paper(nt, tgt, md, out, st);
    FMM_CHECK(cudaGetLastError());
    FMM_CHECK(cudaStreamSynchronize(st));
  } catch (FmmError& e) {
    h->err = e.msg;
    return e.code;
  }
  return FMM_OK;
}
