// Oracle-side Philox4x32-10 counter-based generator (test infrastructure only).
//
// Definition: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
// 1, 2, 3" (SC'11), the Philox-4x32 bijection with 10 rounds.  The paper under
// study uses one stateful generator per thread; a counter-based generator keyed
// by (seed, event, step, slot, purpose) makes every draw reproducible from its
// index, which is what lets the serial oracle and the event-parallel GPU path
// consume identical random numbers (the "identical random numbers give
// identical events" check of Sec. 3.1).
//
// This file is written independently of the CUDA path and shares nothing with
// it; the only common ground is the published definition above.
#pragma once
#include <cstdint>

namespace oracle {

struct Draw4 {
  uint32_t w[4];
};

// One Philox4x32-10 evaluation.  ctr = 128-bit counter, key = 64-bit key.
inline Draw4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                           uint32_t k0, uint32_t k1) {
  const uint32_t kMul0 = 0xD2511F53u;   // round multipliers
  const uint32_t kMul1 = 0xCD9E8D57u;
  const uint32_t kWeyl0 = 0x9E3779B9u;  // key schedule increments
  const uint32_t kWeyl1 = 0xBB67AE85u;
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += kWeyl0;
      k1 += kWeyl1;
    }
    const uint64_t prod0 = static_cast<uint64_t>(kMul0) * c0;
    const uint64_t prod1 = static_cast<uint64_t>(kMul1) * c2;
    const uint32_t hi0 = static_cast<uint32_t>(prod0 >> 32);
    const uint32_t lo0 = static_cast<uint32_t>(prod0);
    const uint32_t hi1 = static_cast<uint32_t>(prod1 >> 32);
    const uint32_t lo1 = static_cast<uint32_t>(prod1);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n1 = lo1;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    const uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  return Draw4{{c0, c1, c2, c3}};
}

// Two 32-bit words -> a double strictly inside (0, 1): the top 26 bits of each
// word form a 52-bit integer m, and u = (m + 1/2) * 2^-52.  Every step is exact
// in binary64, so u never equals 0 or 1.
inline double unit_double(uint32_t hi, uint32_t lo) {
  const uint64_t m = (static_cast<uint64_t>(hi >> 6) << 26) | static_cast<uint64_t>(lo >> 6);
  return (static_cast<double>(m) + 0.5) * 0x1p-52;
}

// Purposes of a draw (fourth counter word).
enum Purpose : uint32_t {
  kPurposeME = 1,      // matrix element: flavour, cos(theta), phi
  kPurposeTrial = 2,   // one trial scale per (dipole, splitting kernel)
  kPurposeWinner = 3,  // z, veto number and azimuth of the winning trial
};

// The pair of uniforms for counter (event, step, slot, purpose) under key seed.
struct UniformPair {
  double u0, u1;
};

inline UniformPair uniform_pair(uint64_t seed, uint32_t event, uint32_t step, uint32_t slot,
                                uint32_t purpose) {
  const Draw4 d = philox4x32_10(event, step, slot, purpose, static_cast<uint32_t>(seed),
                                static_cast<uint32_t>(seed >> 32));
  return UniformPair{unit_double(d.w[0], d.w[1]), unit_double(d.w[2], d.w[3])};
}

}  // namespace oracle
