// field.cuh -- prime-field arithmetic on 8 x 32-bit limbs for sm_103a.
//
// Elements are 256-bit little-endian limb vectors in Montgomery form
// (X = x * 2^256 mod r), as the paper describes field elements: word-sized
// limbs (Section II), results of every field operation in [0, r).
//
// * mul: Montgomery product X * Y * 2^-256 mod r, coarsely integrated operand
//   scanning (CIOS): for each limb b_i, t += a * b_i, then m = t_0 * r' and
//   t = (t + m * r) / 2^32.  The paper finds FF_mul to be the dominant cost of
//   the NTT (Section IV-B: FF_mul + FF_sqr are 93.8% of NTT time) and the
//   32-bit multiply-add (IMAD) the dominant instruction (Section IV-B-2).  Every
//   carry chain is a single asm statement of add.cc / addc.cc instructions, so
//   the carry flag never has to survive between statements.  For r < 2^255
//   (all three fields here) the running value t stays below 2r after each outer
//   step, so nine limbs suffice and no tenth carry limb is kept.
// * add / sub: the paper measures the conditional-reduction branches as 70.5%
//   of FF_add latency (Section IV-B-1) and 52-56% branch efficiency (Section
//   IV-C).  Here both candidates are computed and one is selected with a mask
//   from the borrow -- no branch.
//
// Field-specific shortcuts:
// * BLS12-381 F_r has r = 1 mod 2^32 and limb 1 of r is 2^32 - 1
//   (r' = 2^32 - 1), so m = -t_0 and the products m r_0, m r_1 reduce to adds
//   (the compiler forms them; BLS12-377 F_r shares r_0 = 1).
// * BN254 F_r has r' = 2^32 - 2^28 - 1 and r_0 = 2^32 - 2^28 + 1, so m and the
//   high word of m r_0 + t_0 come from shifts and adds: one wide multiply-add
//   and one multiply fewer per reduction row on the heavy FMA pipe (NTT 2^24:
//   3502 -> 3549 Melem/s).
#pragma once
#include <cstdint>

namespace zkntt {

struct FrBLS12_381 {
    static constexpr uint32_t P0 = 0x00000001u, P1 = 0xffffffffu, P2 = 0xfffe5bfeu, P3 = 0x53bda402u,
                              P4 = 0x09a1d805u, P5 = 0x3339d808u, P6 = 0x299d7d48u, P7 = 0x73eda753u;
    static constexpr uint32_t RP = 0xffffffffu;  // -r^-1 mod 2^32
    static constexpr int ID = 0;
};

struct FrBN254 {
    static constexpr uint32_t P0 = 0xf0000001u, P1 = 0x43e1f593u, P2 = 0x79b97091u, P3 = 0x2833e848u,
                              P4 = 0x8181585du, P5 = 0xb85045b6u, P6 = 0xe131a029u, P7 = 0x30644e72u;
    static constexpr uint32_t RP = 0xefffffffu;
    static constexpr int ID = 1;
};

// BLS12-377 F_r (253 bits; r = 1 mod 2^32 as for BLS12-381, so m = -t_0)
struct FrBLS12_377 {
    static constexpr uint32_t P0 = 0x00000001u, P1 = 0x0a118000u, P2 = 0xd0000001u, P3 = 0x59aa76feu,
                              P4 = 0x5c37b001u, P5 = 0x60b44d1eu, P6 = 0x9a2ca556u, P7 = 0x12ab655eu;
    static constexpr uint32_t RP = 0xffffffffu;
    static constexpr int ID = 2;
};

// ---------------------------------------------------------------------------
// conditional subtraction of r: x in [0, 2r) -> [0, r), branch-free
template <class F>
__device__ __forceinline__ void reduce_once(uint32_t x[8]) {
    uint32_t u[8], mask;
    asm("sub.cc.u32  %0, %9, %17;\n\t"
        "subc.cc.u32 %1, %10, %18;\n\t"
        "subc.cc.u32 %2, %11, %19;\n\t"
        "subc.cc.u32 %3, %12, %20;\n\t"
        "subc.cc.u32 %4, %13, %21;\n\t"
        "subc.cc.u32 %5, %14, %22;\n\t"
        "subc.cc.u32 %6, %15, %23;\n\t"
        "subc.cc.u32 %7, %16, %24;\n\t"
        "subc.u32    %8, 0, 0;"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
          "=r"(u[7]), "=r"(mask)
        : "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(x[5]), "r"(x[6]), "r"(x[7]),
          "n"(F::P0), "n"(F::P1), "n"(F::P2), "n"(F::P3), "n"(F::P4), "n"(F::P5), "n"(F::P6),
          "n"(F::P7));
    // mask = all ones when x < r (borrow): keep x, else take x - r
#pragma unroll
    for (int i = 0; i < 8; i++) x[i] = u[i] ^ ((x[i] ^ u[i]) & mask);
}

// r = a + b mod p, inputs canonical
template <class F>
__device__ __forceinline__ void add(uint32_t r[8], const uint32_t a[8], const uint32_t b[8]) {
    asm("add.cc.u32  %0, %8, %16;\n\t"
        "addc.cc.u32 %1, %9, %17;\n\t"
        "addc.cc.u32 %2, %10, %18;\n\t"
        "addc.cc.u32 %3, %11, %19;\n\t"
        "addc.cc.u32 %4, %12, %20;\n\t"
        "addc.cc.u32 %5, %13, %21;\n\t"
        "addc.cc.u32 %6, %14, %22;\n\t"
        "addc.u32    %7, %15, %23;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]),
          "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
    reduce_once<F>(r);  // a + b < 2r < 2^256: no carry out of limb 7
}

// r = a - b mod p, inputs canonical
template <class F>
__device__ __forceinline__ void sub(uint32_t r[8], const uint32_t a[8], const uint32_t b[8]) {
    uint32_t mask;
    asm("sub.cc.u32  %0, %9, %17;\n\t"
        "subc.cc.u32 %1, %10, %18;\n\t"
        "subc.cc.u32 %2, %11, %19;\n\t"
        "subc.cc.u32 %3, %12, %20;\n\t"
        "subc.cc.u32 %4, %13, %21;\n\t"
        "subc.cc.u32 %5, %14, %22;\n\t"
        "subc.cc.u32 %6, %15, %23;\n\t"
        "subc.cc.u32 %7, %16, %24;\n\t"
        "subc.u32    %8, 0, 0;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(mask)
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]),
          "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
    // on borrow add r back (mask selects the modulus limbs)
    asm("add.cc.u32  %0, %0, %8;\n\t"
        "addc.cc.u32 %1, %1, %9;\n\t"
        "addc.cc.u32 %2, %2, %10;\n\t"
        "addc.cc.u32 %3, %3, %11;\n\t"
        "addc.cc.u32 %4, %4, %12;\n\t"
        "addc.cc.u32 %5, %5, %13;\n\t"
        "addc.cc.u32 %6, %6, %14;\n\t"
        "addc.u32    %7, %7, %15;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
          "+r"(r[7])
        : "r"(F::P0 & mask), "r"(F::P1 & mask), "r"(F::P2 & mask), "r"(F::P3 & mask),
          "r"(F::P4 & mask), "r"(F::P5 & mask), "r"(F::P6 & mask), "r"(F::P7 & mask));
}

// r = a + p - b, in (0, 2p) and congruent to a - b, for canonical a, b: no
// conditional correction.  Only for values that feed mul as its second
// (limb-scanned) operand, which may be any value below 2^256.
template <class F>
__device__ __forceinline__ void sub_lazy(uint32_t r[8], const uint32_t a[8], const uint32_t b[8]) {
    // r = a + p into fresh registers (a stays live for the caller: no copy),
    // then r -= b in place
    asm("add.cc.u32  %0, %8, %16;\n\t"
        "addc.cc.u32 %1, %9, %17;\n\t"
        "addc.cc.u32 %2, %10, %18;\n\t"
        "addc.cc.u32 %3, %11, %19;\n\t"
        "addc.cc.u32 %4, %12, %20;\n\t"
        "addc.cc.u32 %5, %13, %21;\n\t"
        "addc.cc.u32 %6, %14, %22;\n\t"
        "addc.u32    %7, %15, %23;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]),
          "n"(F::P0), "n"(F::P1), "n"(F::P2), "n"(F::P3), "n"(F::P4), "n"(F::P5), "n"(F::P6),
          "n"(F::P7));
    asm("sub.cc.u32  %0, %0, %8;\n\t"
        "subc.cc.u32 %1, %1, %9;\n\t"
        "subc.cc.u32 %2, %2, %10;\n\t"
        "subc.cc.u32 %3, %3, %11;\n\t"
        "subc.cc.u32 %4, %4, %12;\n\t"
        "subc.cc.u32 %5, %5, %13;\n\t"
        "subc.cc.u32 %6, %6, %14;\n\t"
        "subc.u32    %7, %7, %15;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
          "+r"(r[7])
        : "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
}

// ---------------------------------------------------------------------------
// Montgomery product, CIOS with one 64-bit partial product per limb pair.
//
// Outer step i adds a * b_i to the running value t (t < 2r, nine limbs): the
// eight wide products P_j = a_j * b_i are independent; two add-with-carry
// chains fold them in (t += P.lo at positions 0..7, then t += P.hi at
// positions 1..8).  The reduction step forms Q_j = m r_j + t_j with
// m = t_0 r' mod 2^32 -- a 64-bit multiply-add that cannot overflow -- and one
// chain merges Q_j.hi with Q_{j+1}.lo; Q_0.lo is zero by the choice of m, so
// that merge also divides by 2^32.
//
// Why this split: on GB300 the wide multiplies run on the heavy FMA datapath
// at half rate, and a multiply-add whose 64-bit addend is a zero-extended
// 32-bit value also needs a move on that datapath, while the add chains run on
// the ALU pipe.  Using the addend form in the reduction rows and in the last
// product row, and plain wide products with two add chains in the others,
// balances the two pipes.  The first product row starts from t = 0, and the
// asm chains are opaque to the compiler, so it gets its own single chain
// instead of adding zeros.  Measured on GB300, BLS12-381 F_r: 58.3 G
// products/s, against 55.7 with every product row in the two-chain form and
// 43 for separate mad.lo.cc / madc.hi.cc chains.  With r < 2^255 (all
// fields) t < 2r holds after every step, so t_8 never carries out.
__device__ __forceinline__ void merge_product_row(uint32_t t[9], const uint64_t P[8]) {
    uint32_t lo[8], hi[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        lo[j] = uint32_t(P[j]);
        hi[j] = uint32_t(P[j] >> 32);
    }
    asm("add.cc.u32  %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, %10;\n\t"
        "addc.cc.u32 %2, %2, %11;\n\t"
        "addc.cc.u32 %3, %3, %12;\n\t"
        "addc.cc.u32 %4, %4, %13;\n\t"
        "addc.cc.u32 %5, %5, %14;\n\t"
        "addc.cc.u32 %6, %6, %15;\n\t"
        "addc.cc.u32 %7, %7, %16;\n\t"
        "addc.u32    %8, %8, 0;\n\t"
        "add.cc.u32  %1, %1, %17;\n\t"
        "addc.cc.u32 %2, %2, %18;\n\t"
        "addc.cc.u32 %3, %3, %19;\n\t"
        "addc.cc.u32 %4, %4, %20;\n\t"
        "addc.cc.u32 %5, %5, %21;\n\t"
        "addc.cc.u32 %6, %6, %22;\n\t"
        "addc.cc.u32 %7, %7, %23;\n\t"
        "addc.u32    %8, %8, %24;"
        : "+r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]),
          "+r"(t[7]), "+r"(t[8])
        : "r"(lo[0]), "r"(lo[1]), "r"(lo[2]), "r"(lo[3]), "r"(lo[4]), "r"(lo[5]), "r"(lo[6]),
          "r"(lo[7]), "r"(hi[0]), "r"(hi[1]), "r"(hi[2]), "r"(hi[3]), "r"(hi[4]), "r"(hi[5]),
          "r"(hi[6]), "r"(hi[7]));
}

// first product row (t = 0 before it): t = P_0.lo, P_0.hi + P_1.lo, ...,
// P_6.hi + P_7.lo, P_7.hi + carry -- one chain, no adds of zero
__device__ __forceinline__ void merge_first_row(uint32_t t[9], const uint64_t P[8]) {
    uint32_t lo[8], hi[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        lo[j] = uint32_t(P[j]);
        hi[j] = uint32_t(P[j] >> 32);
    }
    t[0] = lo[0];
    asm("add.cc.u32  %0, %8, %16;\n\t"
        "addc.cc.u32 %1, %9, %17;\n\t"
        "addc.cc.u32 %2, %10, %18;\n\t"
        "addc.cc.u32 %3, %11, %19;\n\t"
        "addc.cc.u32 %4, %12, %20;\n\t"
        "addc.cc.u32 %5, %13, %21;\n\t"
        "addc.cc.u32 %6, %14, %22;\n\t"
        "addc.u32    %7, %15, 0;"
        : "=r"(t[1]), "=r"(t[2]), "=r"(t[3]), "=r"(t[4]), "=r"(t[5]), "=r"(t[6]), "=r"(t[7]),
          "=r"(t[8])
        : "r"(hi[0]), "r"(hi[1]), "r"(hi[2]), "r"(hi[3]), "r"(hi[4]), "r"(hi[5]), "r"(hi[6]),
          "r"(hi[7]), "r"(lo[1]), "r"(lo[2]), "r"(lo[3]), "r"(lo[4]), "r"(lo[5]), "r"(lo[6]),
          "r"(lo[7]));
}

// addend-form product merge: with P_j = a_j b_i + t_j,
// t = P_0.lo, P_0.hi + P_1.lo, ..., P_6.hi + P_7.lo, P_7.hi + t_8
__device__ __forceinline__ void merge_addend_row(uint32_t t[9], const uint64_t P[8]) {
    uint32_t lo[8], hi[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        lo[j] = uint32_t(P[j]);
        hi[j] = uint32_t(P[j] >> 32);
    }
    t[0] = lo[0];
    asm("add.cc.u32  %0, %8, %16;\n\t"
        "addc.cc.u32 %1, %9, %17;\n\t"
        "addc.cc.u32 %2, %10, %18;\n\t"
        "addc.cc.u32 %3, %11, %19;\n\t"
        "addc.cc.u32 %4, %12, %20;\n\t"
        "addc.cc.u32 %5, %13, %21;\n\t"
        "addc.cc.u32 %6, %14, %22;\n\t"
        "addc.u32    %7, %15, %7;"
        : "=r"(t[1]), "=r"(t[2]), "=r"(t[3]), "=r"(t[4]), "=r"(t[5]), "=r"(t[6]), "=r"(t[7]),
          "+r"(t[8])
        : "r"(hi[0]), "r"(hi[1]), "r"(hi[2]), "r"(hi[3]), "r"(hi[4]), "r"(hi[5]), "r"(hi[6]),
          "r"(hi[7]), "r"(lo[1]), "r"(lo[2]), "r"(lo[3]), "r"(lo[4]), "r"(lo[5]), "r"(lo[6]),
          "r"(lo[7]));
}

// reduction merge: t'_j = Q_j.hi + Q_{j+1}.lo (j < 7), t'_7 = Q_7.hi + t_8
__device__ __forceinline__ void merge_reduce(uint32_t t[9], const uint64_t Q[8]) {
    uint32_t lo[8], hi[8];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        lo[j] = uint32_t(Q[j]);
        hi[j] = uint32_t(Q[j] >> 32);
    }
    const uint32_t t8 = t[8];
    asm("add.cc.u32  %0, %8, %15;\n\t"
        "addc.cc.u32 %1, %9, %16;\n\t"
        "addc.cc.u32 %2, %10, %17;\n\t"
        "addc.cc.u32 %3, %11, %18;\n\t"
        "addc.cc.u32 %4, %12, %19;\n\t"
        "addc.cc.u32 %5, %13, %20;\n\t"
        "addc.cc.u32 %6, %14, %21;\n\t"
        "addc.u32    %7, %22, %23;"
        : "=r"(t[0]), "=r"(t[1]), "=r"(t[2]), "=r"(t[3]), "=r"(t[4]), "=r"(t[5]), "=r"(t[6]),
          "=r"(t[7])
        : "r"(hi[0]), "r"(hi[1]), "r"(hi[2]), "r"(hi[3]), "r"(hi[4]), "r"(hi[5]), "r"(hi[6]),
          "r"(lo[1]), "r"(lo[2]), "r"(lo[3]), "r"(lo[4]), "r"(lo[5]), "r"(lo[6]), "r"(lo[7]),
          "r"(hi[7]), "r"(t8));
    t[8] = 0;
}

// Product-row / reduction-row forms (build-time choice, see the comment above):
//   0: the first product row is a single chain (t = 0 before it), product rows
//      1..6 without addend, the last product row and every reduction row with
//      the 64-bit addend (shipped)
//   1: neither row uses the addend (all merging on the ALU pipe)
//   2: every row uses the addend
//   4: as 0, with every 64-bit addend formed as the pair {t_j, z_j}, where the
//      z_j are zero words read from constant memory (kept in registers across
//      products) rather than a zero-extension of t_j (build-time option)
#ifndef ZKNTT_MUL_FORM
#define ZKNTT_MUL_FORM 0
#endif

#if ZKNTT_MUL_FORM == 4
// zero words; the product uses them as the high halves of its 64-bit addends
__constant__ uint32_t kAddendHigh[8];
#endif

// a b + {hi, lo} as one 32 x 32 + 64-bit multiply-add
__device__ __forceinline__ uint64_t mad_wide_pair(uint32_t a, uint32_t b, uint32_t lo, uint32_t hi) {
    uint64_t r;
    asm("{\n\t.reg .u64 c;\n\tmov.b64 c, {%3, %4};\n\tmad.wide.u32 %0, %1, %2, c;\n\t}"
        : "=l"(r)
        : "r"(a), "r"(b), "r"(lo), "r"(hi));
    return r;
}

// a b + t (64-bit result) in the addend rows of the product
__device__ __forceinline__ uint64_t addend_mad(uint32_t a, uint32_t b, uint32_t t, uint32_t zh) {
#if ZKNTT_MUL_FORM == 4
    return mad_wide_pair(a, b, t, zh);
#else
    (void)zh;
    return uint64_t(a) * b + t;
#endif
}

// ---------------------------------------------------------------------------
// Form 3 (build-time option, not the default): one level of Karatsuba for the
// 256 x 256-bit product, then a separated-operand-scanning reduction.  The
// paper suggests trading IMAD for IADD3-class work (Section IV-B-2); with
// a = aL + 2^128 aH and b = bL + 2^128 bH the product takes three 4 x 4 limb
// products (48 wide multiplies instead of 64):
//   a b = LL + 2^128 (M - LL - HH) + 2^256 HH,
//   LL = aL bL, HH = aH bH, M = (aL + aH)(bL + bH),
// where the sums carry one bit each, corrected by masked adds.

// z = x * y for 4-limb x, y (8 limbs)
__device__ __forceinline__ void mul4x4(uint32_t z[8], const uint32_t x[4], const uint32_t y[4]) {
    uint64_t P[4];
#pragma unroll
    for (int j = 0; j < 4; j++) P[j] = uint64_t(x[j]) * y[0];
    z[0] = uint32_t(P[0]);
    asm("add.cc.u32  %0, %4, %5;\n\t"
        "addc.cc.u32 %1, %6, %7;\n\t"
        "addc.cc.u32 %2, %8, %9;\n\t"
        "addc.u32    %3, %10, 0;"
        : "=r"(z[1]), "=r"(z[2]), "=r"(z[3]), "=r"(z[4])
        : "r"(uint32_t(P[0] >> 32)), "r"(uint32_t(P[1])), "r"(uint32_t(P[1] >> 32)),
          "r"(uint32_t(P[2])), "r"(uint32_t(P[2] >> 32)), "r"(uint32_t(P[3])),
          "r"(uint32_t(P[3] >> 32)));
#pragma unroll
    for (int i = 1; i < 4; i++) {
#pragma unroll
        for (int j = 0; j < 4; j++) P[j] = uint64_t(x[j]) * y[i];
        uint32_t top;
        asm("add.cc.u32  %0, %0, %5;\n\t"
            "addc.cc.u32 %1, %1, %6;\n\t"
            "addc.cc.u32 %2, %2, %7;\n\t"
            "addc.cc.u32 %3, %3, %8;\n\t"
            "addc.u32    %4, 0, 0;\n\t"
            "add.cc.u32  %1, %1, %9;\n\t"
            "addc.cc.u32 %2, %2, %10;\n\t"
            "addc.cc.u32 %3, %3, %11;\n\t"
            "addc.u32    %4, %4, %12;"
            : "+r"(z[i]), "+r"(z[i + 1]), "+r"(z[i + 2]), "+r"(z[i + 3]), "=r"(top)
            : "r"(uint32_t(P[0])), "r"(uint32_t(P[1])), "r"(uint32_t(P[2])), "r"(uint32_t(P[3])),
              "r"(uint32_t(P[0] >> 32)), "r"(uint32_t(P[1] >> 32)), "r"(uint32_t(P[2] >> 32)),
              "r"(uint32_t(P[3] >> 32)));
        z[i + 4] = top;
    }
}


// Form 3's product: T = a b (16 limbs) by one Karatsuba level, then eight
// word reductions T <- (T + m r 2^(32 i)) with m = T_i r' mod 2^32; the carry
// out of each row's top limb is added to the next row's top limb.  a must be
// canonical (so aH < 2^127), b may be any value below 2^256; T < r 2^256, so
// the result is below 2r and one conditional subtraction canonicalises it.
template <class F>
__device__ __forceinline__ void mul_karatsuba(uint32_t r[8], const uint32_t a[8], const uint32_t b[8]) {
    const uint32_t P[8] = {F::P0, F::P1, F::P2, F::P3, F::P4, F::P5, F::P6, F::P7};
    uint32_t LL[8], HH[8], M[9], sa[4], sb[4], ca, cb;
    mul4x4(LL, a, b);
    mul4x4(HH, a + 4, b + 4);
    asm("add.cc.u32  %0, %5, %9;\n\t"
        "addc.cc.u32 %1, %6, %10;\n\t"
        "addc.cc.u32 %2, %7, %11;\n\t"
        "addc.cc.u32 %3, %8, %12;\n\t"
        "addc.u32    %4, 0, 0;"
        : "=r"(sa[0]), "=r"(sa[1]), "=r"(sa[2]), "=r"(sa[3]), "=r"(ca)
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]));
    asm("add.cc.u32  %0, %5, %9;\n\t"
        "addc.cc.u32 %1, %6, %10;\n\t"
        "addc.cc.u32 %2, %7, %11;\n\t"
        "addc.cc.u32 %3, %8, %12;\n\t"
        "addc.u32    %4, 0, 0;"
        : "=r"(sb[0]), "=r"(sb[1]), "=r"(sb[2]), "=r"(sb[3]), "=r"(cb)
        : "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
    mul4x4(M, sa, sb);
    // M += 2^128 (ca sb + cb sa) + 2^256 ca cb
    const uint32_t ma = 0u - ca, mb = 0u - cb;
    asm("add.cc.u32  %0, %0, %5;\n\t"
        "addc.cc.u32 %1, %1, %6;\n\t"
        "addc.cc.u32 %2, %2, %7;\n\t"
        "addc.cc.u32 %3, %3, %8;\n\t"
        "addc.u32    %4, 0, 0;\n\t"
        "add.cc.u32  %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, %10;\n\t"
        "addc.cc.u32 %2, %2, %11;\n\t"
        "addc.cc.u32 %3, %3, %12;\n\t"
        "addc.u32    %4, %4, %13;"
        : "+r"(M[4]), "+r"(M[5]), "+r"(M[6]), "+r"(M[7]), "=r"(M[8])
        : "r"(sb[0] & ma), "r"(sb[1] & ma), "r"(sb[2] & ma), "r"(sb[3] & ma),
          "r"(sa[0] & mb), "r"(sa[1] & mb), "r"(sa[2] & mb), "r"(sa[3] & mb), "r"(ca & cb));
    // M -= LL, M -= HH (the middle term aL bH + aH bL >= 0)
    asm("sub.cc.u32  %0, %0, %9;\n\t"
        "subc.cc.u32 %1, %1, %10;\n\t"
        "subc.cc.u32 %2, %2, %11;\n\t"
        "subc.cc.u32 %3, %3, %12;\n\t"
        "subc.cc.u32 %4, %4, %13;\n\t"
        "subc.cc.u32 %5, %5, %14;\n\t"
        "subc.cc.u32 %6, %6, %15;\n\t"
        "subc.cc.u32 %7, %7, %16;\n\t"
        "subc.u32    %8, %8, 0;\n\t"
        "sub.cc.u32  %0, %0, %17;\n\t"
        "subc.cc.u32 %1, %1, %18;\n\t"
        "subc.cc.u32 %2, %2, %19;\n\t"
        "subc.cc.u32 %3, %3, %20;\n\t"
        "subc.cc.u32 %4, %4, %21;\n\t"
        "subc.cc.u32 %5, %5, %22;\n\t"
        "subc.cc.u32 %6, %6, %23;\n\t"
        "subc.cc.u32 %7, %7, %24;\n\t"
        "subc.u32    %8, %8, 0;"
        : "+r"(M[0]), "+r"(M[1]), "+r"(M[2]), "+r"(M[3]), "+r"(M[4]), "+r"(M[5]), "+r"(M[6]),
          "+r"(M[7]), "+r"(M[8])
        : "r"(LL[0]), "r"(LL[1]), "r"(LL[2]), "r"(LL[3]), "r"(LL[4]), "r"(LL[5]), "r"(LL[6]),
          "r"(LL[7]), "r"(HH[0]), "r"(HH[1]), "r"(HH[2]), "r"(HH[3]), "r"(HH[4]), "r"(HH[5]),
          "r"(HH[6]), "r"(HH[7]));
    // T = LL + 2^128 M + 2^256 HH
    uint32_t T[16];
#pragma unroll
    for (int i = 0; i < 4; i++) T[i] = LL[i];
    asm("add.cc.u32  %0, %12, %20;\n\t"
        "addc.cc.u32 %1, %13, %21;\n\t"
        "addc.cc.u32 %2, %14, %22;\n\t"
        "addc.cc.u32 %3, %15, %23;\n\t"
        "addc.cc.u32 %4, %16, %24;\n\t"
        "addc.cc.u32 %5, %17, %25;\n\t"
        "addc.cc.u32 %6, %18, %26;\n\t"
        "addc.cc.u32 %7, %19, %27;\n\t"
        "addc.cc.u32 %8, %28, %29;\n\t"
        "addc.cc.u32 %9, %30, 0;\n\t"
        "addc.cc.u32 %10, %31, 0;\n\t"
        "addc.u32    %11, %32, 0;"
        : "=r"(T[4]), "=r"(T[5]), "=r"(T[6]), "=r"(T[7]), "=r"(T[8]), "=r"(T[9]), "=r"(T[10]),
          "=r"(T[11]), "=r"(T[12]), "=r"(T[13]), "=r"(T[14]), "=r"(T[15])
        : "r"(LL[4]), "r"(LL[5]), "r"(LL[6]), "r"(LL[7]), "r"(HH[0]), "r"(HH[1]), "r"(HH[2]),
          "r"(HH[3]), "r"(M[0]), "r"(M[1]), "r"(M[2]), "r"(M[3]), "r"(M[4]), "r"(M[5]), "r"(M[6]),
          "r"(M[7]), "r"(HH[4]), "r"(M[8]), "r"(HH[5]), "r"(HH[6]), "r"(HH[7]));
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        uint32_t m;
        if constexpr (F::RP == 0xefffffffu) m = 0u - T[i] - (T[i] << 28);
        else m = T[i] * F::RP;
        uint64_t X[8];
#pragma unroll
        for (int j = 0; j < 8; j++) X[j] = uint64_t(m) * P[j] + T[i + j];
        if constexpr (F::P0 == 0xf0000001u) {
            uint32_t s0, cy;
            asm("add.cc.u32 %0, %2, %3;\n\t"
                "addc.u32   %1, 0, 0;"
                : "=r"(s0), "=r"(cy)
                : "r"(m), "r"(T[i]));
            X[0] = uint64_t(m - (m >> 4) + cy) << 32;
        }
        uint32_t cn;
        asm("add.cc.u32  %0, %9, %17;\n\t"
            "addc.cc.u32 %1, %10, %18;\n\t"
            "addc.cc.u32 %2, %11, %19;\n\t"
            "addc.cc.u32 %3, %12, %20;\n\t"
            "addc.cc.u32 %4, %13, %21;\n\t"
            "addc.cc.u32 %5, %14, %22;\n\t"
            "addc.cc.u32 %6, %15, %23;\n\t"
            "addc.cc.u32 %7, %16, %7;\n\t"
            "addc.u32    %8, 0, 0;\n\t"
            "add.cc.u32  %7, %7, %24;\n\t"
            "addc.u32    %8, %8, 0;"
            : "=r"(T[i + 1]), "=r"(T[i + 2]), "=r"(T[i + 3]), "=r"(T[i + 4]), "=r"(T[i + 5]),
              "=r"(T[i + 6]), "=r"(T[i + 7]), "+r"(T[i + 8]), "=r"(cn)
            : "r"(uint32_t(X[0] >> 32)), "r"(uint32_t(X[1] >> 32)), "r"(uint32_t(X[2] >> 32)),
              "r"(uint32_t(X[3] >> 32)), "r"(uint32_t(X[4] >> 32)), "r"(uint32_t(X[5] >> 32)),
              "r"(uint32_t(X[6] >> 32)), "r"(uint32_t(X[7] >> 32)), "r"(uint32_t(X[1])),
              "r"(uint32_t(X[2])), "r"(uint32_t(X[3])), "r"(uint32_t(X[4])), "r"(uint32_t(X[5])),
              "r"(uint32_t(X[6])), "r"(uint32_t(X[7])), "r"(c));
        c = cn;
    }
    uint32_t t[8];
#pragma unroll
    for (int i = 0; i < 8; i++) t[i] = T[8 + i];
    reduce_once<F>(t);
#pragma unroll
    for (int i = 0; i < 8; i++) r[i] = t[i];
}

// r = a * b * 2^-256 mod p, canonical.  a must be canonical; b may be any
// value below 2^256: with t <= 2r - 1, a <= r - 1 and b_i, m <= 2^32 - 1 an
// outer step gives (t + a b_i + m r) / 2^32 <= 2r - 1 whatever b is, and the
// final value is below r b / 2^256 + r < 2r, so one conditional subtraction
// canonicalises it.  r may alias a or b.
template <class F>
__device__ __forceinline__ void mul(uint32_t r[8], const uint32_t a[8], const uint32_t b[8]) {
    if constexpr (ZKNTT_MUL_FORM == 3) {
        mul_karatsuba<F>(r, a, b);
        return;
    }
    const uint32_t P[8] = {F::P0, F::P1, F::P2, F::P3, F::P4, F::P5, F::P6, F::P7};
    uint32_t bb[8];
#pragma unroll
    for (int i = 0; i < 8; i++) bb[i] = b[i];
    uint32_t t[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    constexpr bool rows0 = ZKNTT_MUL_FORM == 0 || ZKNTT_MUL_FORM == 4;
    uint32_t zh[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#if ZKNTT_MUL_FORM == 4
#pragma unroll
    for (int j = 0; j < 8; j++) zh[j] = kAddendHigh[j];
#endif
#pragma unroll
    for (int i = 0; i < 8; i++) {
        uint64_t X[8];
        if (rows0 && i == 0) {
#pragma unroll
            for (int j = 0; j < 8; j++) X[j] = uint64_t(a[j]) * bb[0];
            merge_first_row(t, X);
        } else if (ZKNTT_MUL_FORM == 2 || (rows0 && i == 7)) {
#pragma unroll
            for (int j = 0; j < 8; j++) X[j] = addend_mad(a[j], bb[i], t[j], zh[j]);
            merge_addend_row(t, X);
        } else {
#pragma unroll
            for (int j = 0; j < 8; j++) X[j] = uint64_t(a[j]) * bb[i];
            merge_product_row(t, X);
        }
        // m = t_0 r' mod 2^32 (for BLS12-381 F_r, r' = 2^32 - 1 and r_0 = 1,
        // r_1 = 2^32 - 1: the compiler turns those products into adds)
        uint32_t m;
        if constexpr (F::RP == 0xefffffffu) m = 0u - t[0] - (t[0] << 28);  // r' = 2^32 - 2^28 - 1
        else m = t[0] * F::RP;
        if (ZKNTT_MUL_FORM == 1) {
#pragma unroll
            for (int j = 0; j < 8; j++) X[j] = uint64_t(m) * P[j];
            merge_product_row(t, X);  // t_0 becomes 0: shift down one limb
#pragma unroll
            for (int j = 0; j < 8; j++) t[j] = t[j + 1];
            t[8] = 0;
        } else {
#pragma unroll
            for (int j = 0; j < 8; j++)
                // (limbs 1 and 2^32 - 1 stay plain C: the compiler forms them without multiplies)
                X[j] = (P[j] == 1u || P[j] == 0xffffffffu) ? uint64_t(m) * P[j] + t[j]
                                                           : addend_mad(m, P[j], t[j], zh[j]);
            if constexpr (F::P0 == 0xf0000001u) {
                // r_0 = 2^32 - 2^28 + 1: the low word of m r_0 + t_0 is zero by
                // the choice of m, and its high word is m - (m >> 4) + carry(m + t_0)
                uint32_t s, c;
                asm("add.cc.u32 %0, %2, %3;\n\t"
                    "addc.u32   %1, 0, 0;"
                    : "=r"(s), "=r"(c)
                    : "r"(m), "r"(t[0]));
                X[0] = uint64_t(m - (m >> 4) + c) << 32;
            }
            merge_reduce(t, X);
        }
    }
    reduce_once<F>(t);
#pragma unroll
    for (int i = 0; i < 8; i++) r[i] = t[i];
}

// Out-of-line Montgomery product for the once-per-element side paths (input
// and output scales, on-the-fly twiddle composition): keeps the unrolled
// kernels small; the butterfly products stay inline.
template <class F>
__device__ __noinline__ void mul_call(uint32_t r[8], const uint32_t a[8], const uint32_t b[8]) {
    mul<F>(r, a, b);
}

// ---------------------------------------------------------------------------
// element load/store: 32 bytes as two 16-byte vectors
__device__ __forceinline__ void ld_elem(uint32_t x[8], const uint4 *p) {
    uint4 lo = p[0], hi = p[1];
    x[0] = lo.x; x[1] = lo.y; x[2] = lo.z; x[3] = lo.w;
    x[4] = hi.x; x[5] = hi.y; x[6] = hi.z; x[7] = hi.w;
}

__device__ __forceinline__ void ldg_elem(uint32_t x[8], const uint4 *p) {
    uint4 lo = __ldg(p), hi = __ldg(p + 1);
    x[0] = lo.x; x[1] = lo.y; x[2] = lo.z; x[3] = lo.w;
    x[4] = hi.x; x[5] = hi.y; x[6] = hi.z; x[7] = hi.w;
}

// L2-coherent load (bypasses L1) for data another block wrote in this launch
__device__ __forceinline__ void ld_elem_cg(uint32_t x[8], const uint4 *p) {
    uint4 lo = __ldcg(p), hi = __ldcg(p + 1);
    x[0] = lo.x; x[1] = lo.y; x[2] = lo.z; x[3] = lo.w;
    x[4] = hi.x; x[5] = hi.y; x[6] = hi.z; x[7] = hi.w;
}

__device__ __forceinline__ void st_elem(uint4 *p, const uint32_t x[8]) {
    p[0] = make_uint4(x[0], x[1], x[2], x[3]);
    p[1] = make_uint4(x[4], x[5], x[6], x[7]);
}

}  // namespace zkntt
