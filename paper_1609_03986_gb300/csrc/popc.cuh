// Population count of a 512-bit XOR (a Hamming distance) split between the logic
// pipe and the population-count pipe (shared by the brute-force and the dense
// CUDA-core matchers).
#pragma once

#include <stdint.h>

namespace latch {

// carry-save adder: a + b + c = 2 h + l, bit by bit
__device__ __forceinline__ void csa(uint32_t& h, uint32_t& l, uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t u = a ^ b;
    h = (a & b) | (u & c);
    l = u ^ c;
}

// half adder: a + b = 2 h + l
__device__ __forceinline__ void hadd(uint32_t& h, uint32_t& l, uint32_t a, uint32_t b) {
    h = a & b;
    l = a ^ b;
}

// Hamming weight of 16 words.  Words 0-7 go through a carry-save adder tree that
// folds them into one word each of weight 1, 2, 4 and 8 (4 population counts for 8),
// words 8-15 through a population count each: the split keeps the logic pipe (the
// tree) and the population-count pipe about equally busy.
__device__ __forceinline__ int popc16(const uint32_t (&x)[16]) {
    uint32_t h0, l0, h1, l1, h2, l2;
    csa(h0, l0, x[0], x[1], x[2]);
    csa(h1, l1, x[3], x[4], x[5]);
    csa(h2, l2, l0, l1, x[6]);  // weight 1: l2, x7; weight 2: h0, h1, h2
    uint32_t c0, ones, f0, t0;
    hadd(c0, ones, l2, x[7]);
    csa(f0, t0, h0, h1, h2);    // weight 2: t0, c0; weight 4: f0
    uint32_t f1, twos, eights, fours;
    hadd(f1, twos, t0, c0);     // weight 4: f0, f1
    hadd(eights, fours, f0, f1);
    const int tree = 8 * __popc(eights) + 4 * __popc(fours) + 2 * __popc(twos) + __popc(ones);
    return tree + (__popc(x[8]) + __popc(x[9])) + (__popc(x[10]) + __popc(x[11])) + (__popc(x[12]) + __popc(x[13])) +
           (__popc(x[14]) + __popc(x[15]));
}

}  // namespace latch
