// aes_bs.cuh -- bitsliced AES-128 (FIPS-197), 32 blocks a thread: the
// comparator form of the private fragment's cipher (Sec. 5.2.1: the private
// fragment is encrypted with AES), measured against the table form of
// aes_tt.cuh.
//
// State: 128 words, word 8 p + b holding bit b of state byte p of the
// thread's 32 blocks (bit j of the word = block j).  SubBytes is a circuit of
// AND and XOR gates applied to the 8 words of a byte position (all 32 blocks
// at once), ShiftRows only renames byte positions, MixColumns is XORs of
// bit planes (xtime shifts planes and folds plane 7 into planes 0, 1, 3, 4),
// AddRoundKey XORs each plane with all-zeros or all-ones.
//
// The S-box circuit is the straight-line program of Boyar and Peralta ("A
// small depth-16 circuit for the AES S-box", SEC 2012): a linear top layer
// of 27 XORs, a GF(2^4)-inversion middle of 34 AND and 29 XOR gates, a linear
// bottom layer of 38 XOR / XNOR gates, 128 gates.  Its four XNOR gates add
// the affine constant 0x63; here they are plain XORs and the constant is
// folded into round keys 1..10 instead (0x63 in every byte is unchanged by
// ShiftRows and MixColumns: 2 ^ 3 ^ 1 ^ 1 = 1), which the host does when it
// slices the key schedule.
#pragma once

#include <cstdint>

namespace frag {
namespace bs {

constexpr int kBlocks = 32;          // blocks a thread
constexpr int kChunkBlocks = 32 * kBlocks; // blocks a warp: base + 32 j + lane

// the sliced key schedule: word b of byte p of round r is all-ones when bit
// b of that round key byte is set (rounds 1..10 with 0x63 folded in)
struct Keys {
    uint32_t w[11][128];
};

// S-box without its affine constant of 8 bit planes: U0 = bit 7 .. U7 = bit
// 0 of the input, S0 = bit 7 .. S7 = bit 0 of the output
__device__ __forceinline__ void sbox(uint32_t U0, uint32_t U1, uint32_t U2, uint32_t U3, uint32_t U4,
                                     uint32_t U5, uint32_t U6, uint32_t U7, uint32_t &S0, uint32_t &S1,
                                     uint32_t &S2, uint32_t &S3, uint32_t &S4, uint32_t &S5, uint32_t &S6,
                                     uint32_t &S7)
{
    // circuit-begin
    const uint32_t T1 = U0 ^ U3;
    const uint32_t T2 = U0 ^ U5;
    const uint32_t T3 = U0 ^ U6;
    const uint32_t T4 = U3 ^ U5;
    const uint32_t T5 = U4 ^ U6;
    const uint32_t T6 = T1 ^ T5;
    const uint32_t T7 = U1 ^ U2;
    const uint32_t T8 = U7 ^ T6;
    const uint32_t T9 = U7 ^ T7;
    const uint32_t T10 = T6 ^ T7;
    const uint32_t T11 = U1 ^ U5;
    const uint32_t T12 = U2 ^ U5;
    const uint32_t T13 = T3 ^ T4;
    const uint32_t T14 = T6 ^ T11;
    const uint32_t T15 = T5 ^ T11;
    const uint32_t T16 = T5 ^ T12;
    const uint32_t T17 = T9 ^ T16;
    const uint32_t T18 = U3 ^ U7;
    const uint32_t T19 = T7 ^ T18;
    const uint32_t T20 = T1 ^ T19;
    const uint32_t T21 = U6 ^ U7;
    const uint32_t T22 = T7 ^ T21;
    const uint32_t T23 = T2 ^ T22;
    const uint32_t T24 = T2 ^ T10;
    const uint32_t T25 = T20 ^ T17;
    const uint32_t T26 = T3 ^ T16;
    const uint32_t T27 = T1 ^ T12;
    const uint32_t D = U7;
    const uint32_t M1 = T13 & T6;
    const uint32_t M2 = T23 & T8;
    const uint32_t M3 = T14 ^ M1;
    const uint32_t M4 = T19 & D;
    const uint32_t M5 = M4 ^ M1;
    const uint32_t M6 = T3 & T16;
    const uint32_t M7 = T22 & T9;
    const uint32_t M8 = T26 ^ M6;
    const uint32_t M9 = T20 & T17;
    const uint32_t M10 = M9 ^ M6;
    const uint32_t M11 = T1 & T15;
    const uint32_t M12 = T4 & T27;
    const uint32_t M13 = M12 ^ M11;
    const uint32_t M14 = T2 & T10;
    const uint32_t M15 = M14 ^ M11;
    const uint32_t M16 = M3 ^ M2;
    const uint32_t M17 = M5 ^ T24;
    const uint32_t M18 = M8 ^ M7;
    const uint32_t M19 = M10 ^ M15;
    const uint32_t M20 = M16 ^ M13;
    const uint32_t M21 = M17 ^ M15;
    const uint32_t M22 = M18 ^ M13;
    const uint32_t M23 = M19 ^ T25;
    const uint32_t M24 = M22 ^ M23;
    const uint32_t M25 = M22 & M20;
    const uint32_t M26 = M21 ^ M25;
    const uint32_t M27 = M20 ^ M21;
    const uint32_t M28 = M23 ^ M25;
    const uint32_t M29 = M28 & M27;
    const uint32_t M30 = M26 & M24;
    const uint32_t M31 = M20 & M23;
    const uint32_t M32 = M27 & M31;
    const uint32_t M33 = M27 ^ M25;
    const uint32_t M34 = M21 & M22;
    const uint32_t M35 = M24 & M34;
    const uint32_t M36 = M24 ^ M25;
    const uint32_t M37 = M21 ^ M29;
    const uint32_t M38 = M32 ^ M33;
    const uint32_t M39 = M23 ^ M30;
    const uint32_t M40 = M35 ^ M36;
    const uint32_t M41 = M38 ^ M40;
    const uint32_t M42 = M37 ^ M39;
    const uint32_t M43 = M37 ^ M38;
    const uint32_t M44 = M39 ^ M40;
    const uint32_t M45 = M42 ^ M41;
    const uint32_t M46 = M44 & T6;
    const uint32_t M47 = M40 & T8;
    const uint32_t M48 = M39 & D;
    const uint32_t M49 = M43 & T16;
    const uint32_t M50 = M38 & T9;
    const uint32_t M51 = M37 & T17;
    const uint32_t M52 = M42 & T15;
    const uint32_t M53 = M45 & T27;
    const uint32_t M54 = M41 & T10;
    const uint32_t M55 = M44 & T13;
    const uint32_t M56 = M40 & T23;
    const uint32_t M57 = M39 & T19;
    const uint32_t M58 = M43 & T3;
    const uint32_t M59 = M38 & T22;
    const uint32_t M60 = M37 & T20;
    const uint32_t M61 = M42 & T1;
    const uint32_t M62 = M45 & T4;
    const uint32_t M63 = M41 & T2;
    const uint32_t L0 = M61 ^ M62;
    const uint32_t L1 = M50 ^ M56;
    const uint32_t L2 = M46 ^ M48;
    const uint32_t L3 = M47 ^ M55;
    const uint32_t L4 = M54 ^ M58;
    const uint32_t L5 = M49 ^ M61;
    const uint32_t L6 = M62 ^ L5;
    const uint32_t L7 = M46 ^ L3;
    const uint32_t L8 = M51 ^ M59;
    const uint32_t L9 = M52 ^ M53;
    const uint32_t L10 = M53 ^ L4;
    const uint32_t L11 = M60 ^ L2;
    const uint32_t L12 = M48 ^ M51;
    const uint32_t L13 = M50 ^ L0;
    const uint32_t L14 = M52 ^ M61;
    const uint32_t L15 = M55 ^ L1;
    const uint32_t L16 = M56 ^ L0;
    const uint32_t L17 = M57 ^ L1;
    const uint32_t L18 = M58 ^ L8;
    const uint32_t L19 = M63 ^ L4;
    const uint32_t L20 = L0 ^ L1;
    const uint32_t L21 = L1 ^ L7;
    const uint32_t L22 = L3 ^ L12;
    const uint32_t L23 = L18 ^ L2;
    const uint32_t L24 = L15 ^ L9;
    const uint32_t L25 = L6 ^ L10;
    const uint32_t L26 = L7 ^ L9;
    const uint32_t L27 = L8 ^ L10;
    const uint32_t L28 = L11 ^ L14;
    const uint32_t L29 = L11 ^ L17;
    S0 = L6 ^ L24;
    S1 = L16 ^ L26;
    S2 = L19 ^ L28;
    S3 = L6 ^ L21;
    S4 = L20 ^ L22;
    S5 = L25 ^ L29;
    S6 = L13 ^ L27;
    S7 = L6 ^ L23;
    // circuit-end
}

// SubBytes and ShiftRows: byte (row, col) of x goes through the S-box to
// byte (row, col - row mod 4) of y
__device__ __forceinline__ void sub_shift(const uint32_t (&x)[128], uint32_t (&y)[128])
{
#pragma unroll
    for (int p = 0; p < 16; ++p) {
        const int row = p & 3, col = p >> 2, q = row + 4 * ((col - row) & 3);
        sbox(x[8 * p + 7], x[8 * p + 6], x[8 * p + 5], x[8 * p + 4], x[8 * p + 3], x[8 * p + 2], x[8 * p + 1],
             x[8 * p + 0], y[8 * q + 7], y[8 * q + 6], y[8 * q + 5], y[8 * q + 4], y[8 * q + 3], y[8 * q + 2],
             y[8 * q + 1], y[8 * q + 0]);
    }
}

// MixColumns: out_i = 2 a_i ^ 3 a_(i+1) ^ a_(i+2) ^ a_(i+3) = a_i ^ (a_0 ^ a_1
// ^ a_2 ^ a_3) ^ xtime(a_i ^ a_(i+1)) for the rows i of each column
__device__ __forceinline__ void mix(const uint32_t (&y)[128], uint32_t (&z)[128])
{
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t al[8];
#pragma unroll
        for (int b = 0; b < 8; ++b)
            al[b] = y[8 * (4 * c) + b] ^ y[8 * (4 * c + 1) + b] ^ y[8 * (4 * c + 2) + b] ^ y[8 * (4 * c + 3) + b];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int p = 4 * c + i, pn = 4 * c + ((i + 1) & 3);
            uint32_t t[8];
#pragma unroll
            for (int b = 0; b < 8; ++b)
                t[b] = y[8 * p + b] ^ y[8 * pn + b];
            const uint32_t xt[8] = {t[7], t[0] ^ t[7], t[1], t[2] ^ t[7], t[3] ^ t[7], t[4], t[5], t[6]};
#pragma unroll
            for (int b = 0; b < 8; ++b)
                z[8 * p + b] = y[8 * p + b] ^ al[b] ^ xt[b];
        }
    }
}

// 32 x 32 bit transpose in place: afterwards bit k of A[j] is what bit j of
// A[k] was
__device__ __forceinline__ void transpose32(uint32_t (&A)[32])
{
    uint32_t m = 0x0000ffffu;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            if ((k & s) == 0) {
                const uint32_t t = ((A[k] >> s) ^ A[k + s]) & m;
                A[k + s] ^= t;
                A[k] ^= t << s;
            }
        }
        m ^= m << (s >> 1);
    }
}

} // namespace bs
} // namespace frag
