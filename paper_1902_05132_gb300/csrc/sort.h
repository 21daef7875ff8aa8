// Device scans and sorts of the tree build and of the M2L scheduling: an
// exclusive prefix sum of ints and a stable least-significant-digit radix
// sort of (64-bit key, int value) pairs, 8 bits per pass.  Run on `st`
// without host synchronization; `tmp` is grown as needed (it may allocate).
#pragma once
#include <cstdint>

#include "fmm_internal.h"

// out[i] = in[0] + ... + in[i-1] (out[0] = 0); in and out may not overlap.
void dev_exclusive_scan(const int* in, int* out, long n, DevBuf& tmp, cudaStream_t st);

// Stable sort of n (key, value) pairs by bits [bit0, bit1) of the keys:
// kout/vout receive the sorted pairs; kin/vin are used as ping-pong buffers
// and are overwritten.  Equal keys keep their input order.
void dev_sort_pairs(unsigned long long* kin, int* vin, unsigned long long* kout, int* vout, long n, int bit0, int bit1, DevBuf& tmp,
                    cudaStream_t st);

// Run-length encoding of sorted keys: ukeys[r], counts[r] for r < *nruns_d
// (device count written on `st`).
void dev_run_length(const unsigned long long* keys, long n, unsigned long long* ukeys, int* counts, int* nruns_d, DevBuf& tmp,
                    cudaStream_t st);
