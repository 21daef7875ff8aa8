// Device scans and sorts (see sort.h).
//
// Scan: each CTA of 256 threads scans 2048 consecutive ints (8 per thread),
// writes its total; the totals are scanned the same way (recursively) and
// added back.
// Sort: per pass of 8 bits, (1) every CTA counts the digits of its tile of
// 1024 pairs, (2) the counts laid out digit-major, [digit][tile], are
// scanned, which gives every (digit, tile) its first output position, (3)
// every CTA ranks its pairs within the tile and scatters them.  Ranking keeps
// the input order: tile item i = w*128 + r*32 + lane is handled by warp w in
// round r, rounds in order; within a round the lanes with the same digit
// find each other with __match_any_sync and count the lower lanes, and a
// per-warp, per-digit counter in shared memory carries the counts of the
// earlier rounds; the warps' counters are then summed in warp order.
#include "sort.h"

#include <algorithm>
#include <vector>

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;     // 2048
constexpr int kSortThreads = 256;
constexpr int kSortTile = 1024;
constexpr int kWarps = kSortThreads / 32;

// Exclusive scan of the per-thread values of a CTA of kScanThreads threads;
// returns the thread's prefix and writes the CTA total to *total.
__device__ inline int block_excl_scan(int v, int* warp_tot, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
    int s = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = s - t;
    if (lane == 31) *total = s;
  }
  __syncthreads();
  return warp_tot[w] + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const int* __restrict__ in, int* __restrict__ out, long n,
                                                           int* __restrict__ sums) {
  __shared__ int warp_tot[32];
  __shared__ int total;
  const long base = (long)blockIdx.x * kScanTile + (long)threadIdx.x * kScanPer;
  int v[kScanPer];
  int s = 0;
#pragma unroll
  for (int j = 0; j < kScanPer; ++j) {
    v[j] = (base + j < n) ? in[base + j] : 0;
    s += v[j];
  }
  int run = block_excl_scan(s, warp_tot, &total);
#pragma unroll
  for (int j = 0; j < kScanPer; ++j) {
    if (base + j < n) out[base + j] = run;
    run += v[j];
  }
  if (threadIdx.x == 0 && sums) sums[blockIdx.x] = total;
}

__global__ void k_scan_add(int* __restrict__ out, long n, const int* __restrict__ offs) {
  const long i = (long)blockIdx.x * kScanTile + threadIdx.x;
  const int add = offs[blockIdx.x];
  for (int j = 0; j < kScanPer; ++j) {
    const long k = i + (long)j * kScanThreads;
    if (k < n) out[k] += add;
  }
}

void scan_rec(const int* in, int* out, long n, int* scratch, cudaStream_t st) {
  const long nb = (n + kScanTile - 1) / kScanTile;
  if (nb <= 1) {
    LAUNCH(k_scan_tile<<<1, kScanThreads, 0, st>>>(in, out, n, nullptr));
    return;
  }
  int* sums = scratch;
  int* sums_scan = scratch + nb;
  LAUNCH(k_scan_tile<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, sums));
  scan_rec(sums, sums_scan, nb, scratch + 2 * nb, st);
  LAUNCH(k_scan_add<<<(unsigned)nb, kScanThreads, 0, st>>>(out, n, sums_scan));
}

long scan_scratch(long n) {
  long tot = 0;
  for (long nb = (n + kScanTile - 1) / kScanTile; nb > 1; nb = (nb + kScanTile - 1) / kScanTile) tot += 2 * nb;
  return tot + 16;
}

// digit counts of every tile: hist[d * ntiles + tile]
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const unsigned long long* __restrict__ keys, long n, int shift,
                                                           int* __restrict__ hist, int ntiles) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const long base = (long)blockIdx.x * kSortTile;
  for (int j = threadIdx.x; j < kSortTile; j += kSortThreads) {
    const long i = base + j;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 0xFF], 1);
  }
  __syncthreads();
  hist[(long)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const unsigned long long* __restrict__ kin,
                                                              const int* __restrict__ vin, unsigned long long* __restrict__ kout,
                                                              int* __restrict__ vout, long n, int shift,
                                                              const int* __restrict__ offs, int ntiles) {
  __shared__ int wcnt[kWarps][256];            // items of each digit seen by each warp so far
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = lane; d < 256; d += 32) wcnt[w][d] = 0;
  __syncwarp();
  const long base = (long)blockIdx.x * kSortTile + (long)w * (kSortTile / kWarps);
  unsigned long long k[4];
  int v[4], dig[4], rank[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const long i = base + r * 32 + lane;
    const bool valid = i < n;
    k[r] = valid ? kin[i] : 0;
    v[r] = valid ? vin[i] : 0;
    dig[r] = valid ? (int)((k[r] >> shift) & 0xFF) : 256 + lane;     // padding: a digit of its own
    const unsigned peers = __match_any_sync(0xffffffffu, dig[r]);
    const int below = __popc(peers & ((1u << lane) - 1u));
    const int leader = __ffs(peers) - 1;
    if (valid) rank[r] = wcnt[w][dig[r]] + below;
    __syncwarp();
    if (valid && lane == leader) wcnt[w][dig[r]] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // prefix over the warps, per digit: the first slot of warp w's items of digit d
  for (int d = threadIdx.x; d < 256; d += kSortThreads) {
    int s = offs[(long)d * ntiles + blockIdx.x];
    for (int ww = 0; ww < kWarps; ++ww) {
      const int c = wcnt[ww][d];
      wcnt[ww][d] = s;
      s += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const long i = base + r * 32 + lane;
    if (i < n) {
      const int pos = wcnt[w][dig[r]] + rank[r];
      kout[pos] = k[r];
      vout[pos] = v[r];
    }
  }
}

__global__ void k_run_flags(const unsigned long long* __restrict__ keys, long n, int* __restrict__ flag) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_run_write(const unsigned long long* __restrict__ keys, long n, const int* __restrict__ flag,
                            const int* __restrict__ pos, unsigned long long* __restrict__ ukeys, int* __restrict__ start,
                            int* __restrict__ nruns) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (flag[i]) {
    ukeys[pos[i]] = keys[i];
    start[pos[i]] = (int)i;
  }
  if (i == n - 1) {
    const int r = pos[i] + flag[i];
    *nruns = r;
    start[r] = (int)n;
  }
}

__global__ void k_run_counts(const int* __restrict__ start, const int* __restrict__ nruns, int* __restrict__ counts,
                             long cap) {
  const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < cap && r < *nruns) counts[r] = start[r + 1] - start[r];
}

}  // namespace

void dev_exclusive_scan(const int* in, int* out, long n, DevBuf& tmp, cudaStream_t st) {
  if (n <= 0) return;
  tmp.ensure(sizeof(int) * (size_t)scan_scratch(n));
  scan_rec(in, out, n, tmp.as<int>(), st);
}

void dev_sort_pairs(unsigned long long* kin, int* vin, unsigned long long* kout, int* vout, long n, int bit0, int bit1, DevBuf& tmp,
                    cudaStream_t st) {
  if (n <= 0) return;
  const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
  const long nh = 256L * ntiles;
  tmp.ensure(sizeof(int) * (size_t)(2 * nh + scan_scratch(nh)));
  int* hist = tmp.as<int>();
  int* offs = hist + nh;
  int* scratch = offs + nh;
  const int npass = (bit1 - bit0 + 7) / 8;
  // passes alternate between the two buffers; an even number of passes
  // would end in kin, so the last pass writes to kout in every case
  unsigned long long* ks = kin;
  int* vs = vin;
  for (int p = 0; p < npass; ++p) {
    const bool last = p == npass - 1;
    unsigned long long* kd = last ? kout : (ks == kin ? kout : kin);
    int* vd = last ? vout : (vs == vin ? vout : vin);
    if (last && ks == kout) {                  // the source is kout itself: go through kin first
      FMM_CHECK(cudaMemcpyAsync(kin, kout, sizeof(unsigned long long) * n, cudaMemcpyDeviceToDevice, st));
      FMM_CHECK(cudaMemcpyAsync(vin, vout, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
      ks = kin;
      vs = vin;
    }
    const int shift = bit0 + 8 * p;
    LAUNCH(k_sort_hist<<<ntiles, kSortThreads, 0, st>>>(ks, n, shift, hist, ntiles));
    scan_rec(hist, offs, nh, scratch, st);
    LAUNCH(k_sort_scatter<<<ntiles, kSortThreads, 0, st>>>(ks, vs, kd, vd, n, shift, offs, ntiles));
    ks = kd;
    vs = vd;
  }
}

void dev_run_length(const unsigned long long* keys, long n, unsigned long long* ukeys, int* counts, int* nruns_d, DevBuf& tmp,
                    cudaStream_t st) {
  if (n <= 0) {
    FMM_CHECK(cudaMemsetAsync(nruns_d, 0, sizeof(int), st));
    return;
  }
  DevBuf* t = &tmp;
  const long scr = scan_scratch(n);
  t->ensure(sizeof(int) * (size_t)(3 * n + 1 + scr));
  int* flag = t->as<int>();
  int* pos = flag + n;
  int* start = pos + n;                       // n + 1 entries
  int* scratch = start + n + 1;
  LAUNCH(k_run_flags<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(keys, n, flag));
  scan_rec(flag, pos, n, scratch, st);
  LAUNCH(k_run_write<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(keys, n, flag, pos, ukeys, start, nruns_d));
  LAUNCH(k_run_counts<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(start, nruns_d, counts, n));
}
