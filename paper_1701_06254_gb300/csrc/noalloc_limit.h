/* Size rule of sim_ls_residual_norm_noalloc, kept in plain C so that it can
 * be checked on a machine without a GPU.
 *
 * The allocation-free residual norm reduces ROWS_PER_BLOCK block rows per
 * thread block into one partial sum held in a fixed device array of
 * MAX_BLOCKS doubles, so it handles at most MAX_BLOCKS * ROWS_PER_BLOCK
 * block rows. */
#ifndef RS_NOALLOC_LIMIT_H
#define RS_NOALLOC_LIMIT_H

#define NOALLOC_ROWS_PER_BLOCK 4096        /* block rows handled by one thread block */
#define NOALLOC_MAX_BLOCKS 4096            /* scratch capacity: one partial per thread block */

/* number of partial sums for nb block rows, or -1 when nb is outside
 * [1, NOALLOC_MAX_BLOCKS * NOALLOC_ROWS_PER_BLOCK] */
static inline long long rs_noalloc_blocks(long long nb)
{
  if (nb < 1) return -1;
  long long m = (nb + NOALLOC_ROWS_PER_BLOCK - 1) / NOALLOC_ROWS_PER_BLOCK;
  return m > NOALLOC_MAX_BLOCKS ? -1 : m;
}

#endif
