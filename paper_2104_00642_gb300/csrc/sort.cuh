// sort.cuh -- stable tile sort (sort.cu).
#pragma once
#include "pic_internal.cuh"
#include "push.cuh"

namespace pic {

size_t sort_scratch_bytes(long long cap);
size_t scan_scratch_words(long long m);
void scan_exclusive(const uint32_t *in, uint32_t *out, long long m, uint32_t *scratch, cudaStream_t st);
void scan_block_sums(const uint32_t *in, long long m, uint32_t *bsum, uint32_t *scratch, cudaStream_t st,
                     const long long *dn = nullptr);
long long scan_blocks(long long m);  // blocks of the scan of m words (kScanItems each)
void sort_by_tile(const uint32_t *cell, long long n, const long long *dcount_in, const Grid &g, void *scratch,
                  uint32_t *starts, long long *dcount_out, const uint32_t **perm, const uint32_t **skeys,
                  cudaStream_t st);
void launch_permute_f32(const PartF32 &src, const PartF32 &dst, const uint32_t *perm, const long long *dcount,
                        long long n, int dim, cudaStream_t st);
void launch_permute_f64(const PartF64 &src, const PartF64 &dst, const uint32_t *perm, const long long *dcount,
                        long long n, int dim, cudaStream_t st);

}  // namespace pic
