// Generated by gen_networks.py: rank-(k*k-1)/2 selection networks.
// Do not edit by hand; rerun the generator.
#pragma once
#include <cstdint>

namespace fnr {

template <int K> struct MedianNet;

// k=3: 20 compare-exchanges, 32 min/max ops
template <> struct MedianNet<3> {
  static constexpr int kOps = 32;
  template <class Op> __device__ __forceinline__ static uint32_t run(uint32_t (&v)[9], Op op) {
    { uint32_t t = op.mn(v[0], v[3]); v[3] = op.mx(v[0], v[3]); v[0] = t; }
    { uint32_t t = op.mn(v[3], v[6]); v[6] = op.mx(v[3], v[6]); v[3] = t; }
    { uint32_t t = op.mn(v[0], v[3]); v[3] = op.mx(v[0], v[3]); v[0] = t; }
    { uint32_t t = op.mn(v[1], v[4]); v[4] = op.mx(v[1], v[4]); v[1] = t; }
    { uint32_t t = op.mn(v[4], v[7]); v[7] = op.mx(v[4], v[7]); v[4] = t; }
    { uint32_t t = op.mn(v[1], v[4]); v[4] = op.mx(v[1], v[4]); v[1] = t; }
    { uint32_t t = op.mn(v[2], v[5]); v[5] = op.mx(v[2], v[5]); v[2] = t; }
    { uint32_t t = op.mn(v[5], v[8]); v[8] = op.mx(v[5], v[8]); v[5] = t; }
    { uint32_t t = op.mn(v[2], v[5]); v[5] = op.mx(v[2], v[5]); v[2] = t; }
    v[1] = op.mx(v[0], v[1]);
    v[2] = op.mx(v[1], v[2]);
    { uint32_t t = op.mn(v[3], v[4]); v[4] = op.mx(v[3], v[4]); v[3] = t; }
    v[4] = op.mn(v[4], v[5]);
    v[4] = op.mx(v[3], v[4]);
    { uint32_t t = op.mn(v[6], v[7]); v[7] = op.mx(v[6], v[7]); v[6] = t; }
    v[7] = op.mn(v[7], v[8]);
    v[6] = op.mn(v[6], v[7]);
    { uint32_t t = op.mn(v[2], v[4]); v[4] = op.mx(v[2], v[4]); v[2] = t; }
    v[4] = op.mn(v[4], v[6]);
    v[4] = op.mx(v[2], v[4]);
    return v[4];
  }
};

// k=5: 113 compare-exchanges, 202 min/max ops
template <> struct MedianNet<5> {
  static constexpr int kOps = 202;
  template <class Op> __device__ __forceinline__ static uint32_t run(uint32_t (&v)[25], Op op) {
    { uint32_t t = op.mn(v[0], v[16]); v[16] = op.mx(v[0], v[16]); v[0] = t; }
    { uint32_t t = op.mn(v[1], v[17]); v[17] = op.mx(v[1], v[17]); v[1] = t; }
    { uint32_t t = op.mn(v[2], v[18]); v[18] = op.mx(v[2], v[18]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[19]); v[19] = op.mx(v[3], v[19]); v[3] = t; }
    { uint32_t t = op.mn(v[4], v[20]); v[20] = op.mx(v[4], v[20]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[21]); v[21] = op.mx(v[5], v[21]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[22]); v[22] = op.mx(v[6], v[22]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[23]); v[23] = op.mx(v[7], v[23]); v[7] = t; }
    { uint32_t t = op.mn(v[8], v[24]); v[24] = op.mx(v[8], v[24]); v[8] = t; }
    { uint32_t t = op.mn(v[0], v[8]); v[8] = op.mx(v[0], v[8]); v[0] = t; }
    { uint32_t t = op.mn(v[1], v[9]); v[9] = op.mx(v[1], v[9]); v[1] = t; }
    { uint32_t t = op.mn(v[2], v[10]); v[10] = op.mx(v[2], v[10]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[11]); v[11] = op.mx(v[3], v[11]); v[3] = t; }
    { uint32_t t = op.mn(v[4], v[12]); v[12] = op.mx(v[4], v[12]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[13]); v[13] = op.mx(v[5], v[13]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[14]); v[14] = op.mx(v[6], v[14]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[15]); v[15] = op.mx(v[7], v[15]); v[7] = t; }
    { uint32_t t = op.mn(v[16], v[24]); v[24] = op.mx(v[16], v[24]); v[16] = t; }
    { uint32_t t = op.mn(v[8], v[16]); v[16] = op.mx(v[8], v[16]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[17]); v[17] = op.mx(v[9], v[17]); v[9] = t; }
    { uint32_t t = op.mn(v[10], v[18]); v[18] = op.mx(v[10], v[18]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[19]); v[19] = op.mx(v[11], v[19]); v[11] = t; }
    { uint32_t t = op.mn(v[12], v[20]); v[20] = op.mx(v[12], v[20]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[21]); v[21] = op.mx(v[13], v[21]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[22]); v[22] = op.mx(v[14], v[22]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[23]); v[23] = op.mx(v[15], v[23]); v[15] = t; }
    { uint32_t t = op.mn(v[0], v[4]); v[4] = op.mx(v[0], v[4]); v[0] = t; }
    { uint32_t t = op.mn(v[1], v[5]); v[5] = op.mx(v[1], v[5]); v[1] = t; }
    { uint32_t t = op.mn(v[2], v[6]); v[6] = op.mx(v[2], v[6]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[7]); v[7] = op.mx(v[3], v[7]); v[3] = t; }
    { uint32_t t = op.mn(v[8], v[12]); v[12] = op.mx(v[8], v[12]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[13]); v[13] = op.mx(v[9], v[13]); v[9] = t; }
    { uint32_t t = op.mn(v[10], v[14]); v[14] = op.mx(v[10], v[14]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[15]); v[15] = op.mx(v[11], v[15]); v[11] = t; }
    { uint32_t t = op.mn(v[16], v[20]); v[20] = op.mx(v[16], v[20]); v[16] = t; }
    { uint32_t t = op.mn(v[17], v[21]); v[21] = op.mx(v[17], v[21]); v[17] = t; }
    { uint32_t t = op.mn(v[18], v[22]); v[22] = op.mx(v[18], v[22]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[23]); v[23] = op.mx(v[19], v[23]); v[19] = t; }
    { uint32_t t = op.mn(v[4], v[16]); v[16] = op.mx(v[4], v[16]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[17]); v[17] = op.mx(v[5], v[17]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[18]); v[18] = op.mx(v[6], v[18]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[19]); v[19] = op.mx(v[7], v[19]); v[7] = t; }
    { uint32_t t = op.mn(v[12], v[24]); v[24] = op.mx(v[12], v[24]); v[12] = t; }
    { uint32_t t = op.mn(v[4], v[8]); v[8] = op.mx(v[4], v[8]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[9]); v[9] = op.mx(v[5], v[9]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[10]); v[10] = op.mx(v[6], v[10]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[11]); v[11] = op.mx(v[7], v[11]); v[7] = t; }
    { uint32_t t = op.mn(v[12], v[16]); v[16] = op.mx(v[12], v[16]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[17]); v[17] = op.mx(v[13], v[17]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[18]); v[18] = op.mx(v[14], v[18]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[19]); v[19] = op.mx(v[15], v[19]); v[15] = t; }
    { uint32_t t = op.mn(v[20], v[24]); v[24] = op.mx(v[20], v[24]); v[20] = t; }
    { uint32_t t = op.mn(v[0], v[2]); v[2] = op.mx(v[0], v[2]); v[0] = t; }
    { uint32_t t = op.mn(v[1], v[3]); v[3] = op.mx(v[1], v[3]); v[1] = t; }
    { uint32_t t = op.mn(v[4], v[6]); v[6] = op.mx(v[4], v[6]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[7]); v[7] = op.mx(v[5], v[7]); v[5] = t; }
    { uint32_t t = op.mn(v[8], v[10]); v[10] = op.mx(v[8], v[10]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[11]); v[11] = op.mx(v[9], v[11]); v[9] = t; }
    { uint32_t t = op.mn(v[12], v[14]); v[14] = op.mx(v[12], v[14]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[15]); v[15] = op.mx(v[13], v[15]); v[13] = t; }
    { uint32_t t = op.mn(v[16], v[18]); v[18] = op.mx(v[16], v[18]); v[16] = t; }
    { uint32_t t = op.mn(v[17], v[19]); v[19] = op.mx(v[17], v[19]); v[17] = t; }
    { uint32_t t = op.mn(v[20], v[22]); v[22] = op.mx(v[20], v[22]); v[20] = t; }
    { uint32_t t = op.mn(v[21], v[23]); v[23] = op.mx(v[21], v[23]); v[21] = t; }
    { uint32_t t = op.mn(v[2], v[16]); v[16] = op.mx(v[2], v[16]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[17]); v[17] = op.mx(v[3], v[17]); v[3] = t; }
    { uint32_t t = op.mn(v[6], v[20]); v[20] = op.mx(v[6], v[20]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[21]); v[21] = op.mx(v[7], v[21]); v[7] = t; }
    { uint32_t t = op.mn(v[10], v[24]); v[24] = op.mx(v[10], v[24]); v[10] = t; }
    { uint32_t t = op.mn(v[2], v[8]); v[8] = op.mx(v[2], v[8]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[9]); v[9] = op.mx(v[3], v[9]); v[3] = t; }
    { uint32_t t = op.mn(v[6], v[12]); v[12] = op.mx(v[6], v[12]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[13]); v[13] = op.mx(v[7], v[13]); v[7] = t; }
    { uint32_t t = op.mn(v[10], v[16]); v[16] = op.mx(v[10], v[16]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[17]); v[17] = op.mx(v[11], v[17]); v[11] = t; }
    { uint32_t t = op.mn(v[14], v[20]); v[20] = op.mx(v[14], v[20]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[21]); v[21] = op.mx(v[15], v[21]); v[15] = t; }
    { uint32_t t = op.mn(v[18], v[24]); v[24] = op.mx(v[18], v[24]); v[18] = t; }
    { uint32_t t = op.mn(v[2], v[4]); v[4] = op.mx(v[2], v[4]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[5]); v[5] = op.mx(v[3], v[5]); v[3] = t; }
    { uint32_t t = op.mn(v[6], v[8]); v[8] = op.mx(v[6], v[8]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[9]); v[9] = op.mx(v[7], v[9]); v[7] = t; }
    { uint32_t t = op.mn(v[10], v[12]); v[12] = op.mx(v[10], v[12]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[13]); v[13] = op.mx(v[11], v[13]); v[11] = t; }
    { uint32_t t = op.mn(v[14], v[16]); v[16] = op.mx(v[14], v[16]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[17]); v[17] = op.mx(v[15], v[17]); v[15] = t; }
    { uint32_t t = op.mn(v[18], v[20]); v[20] = op.mx(v[18], v[20]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[21]); v[21] = op.mx(v[19], v[21]); v[19] = t; }
    { uint32_t t = op.mn(v[22], v[24]); v[24] = op.mx(v[22], v[24]); v[22] = t; }
    v[1] = op.mx(v[0], v[1]);
    v[3] = op.mx(v[2], v[3]);
    v[5] = op.mx(v[4], v[5]);
    v[7] = op.mx(v[6], v[7]);
    v[9] = op.mx(v[8], v[9]);
    v[11] = op.mx(v[10], v[11]);
    v[12] = op.mn(v[12], v[13]);
    v[14] = op.mn(v[14], v[15]);
    v[16] = op.mn(v[16], v[17]);
    v[18] = op.mn(v[18], v[19]);
    v[20] = op.mn(v[20], v[21]);
    v[22] = op.mn(v[22], v[23]);
    v[16] = op.mx(v[1], v[16]);
    v[18] = op.mx(v[3], v[18]);
    v[5] = op.mn(v[5], v[20]);
    v[7] = op.mn(v[7], v[22]);
    v[9] = op.mn(v[9], v[24]);
    v[12] = op.mx(v[5], v[12]);
    v[14] = op.mx(v[7], v[14]);
    v[9] = op.mn(v[9], v[16]);
    v[11] = op.mn(v[11], v[18]);
    v[12] = op.mx(v[9], v[12]);
    v[11] = op.mn(v[11], v[14]);
    v[12] = op.mx(v[11], v[12]);
    return v[12];
  }
};

// k=7: 313 compare-exchanges, 578 min/max ops
template <> struct MedianNet<7> {
  static constexpr int kOps = 578;
  template <class Op> __device__ __forceinline__ static uint32_t run(uint32_t (&v)[49], Op op) {
    { uint32_t t = op.mn(v[0], v[32]); v[32] = op.mx(v[0], v[32]); v[0] = t; }
    { uint32_t t = op.mn(v[1], v[33]); v[33] = op.mx(v[1], v[33]); v[1] = t; }
    { uint32_t t = op.mn(v[2], v[34]); v[34] = op.mx(v[2], v[34]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[35]); v[35] = op.mx(v[3], v[35]); v[3] = t; }
    { uint32_t t = op.mn(v[4], v[36]); v[36] = op.mx(v[4], v[36]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[37]); v[37] = op.mx(v[5], v[37]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[38]); v[38] = op.mx(v[6], v[38]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[39]); v[39] = op.mx(v[7], v[39]); v[7] = t; }
    { uint32_t t = op.mn(v[8], v[40]); v[40] = op.mx(v[8], v[40]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[41]); v[41] = op.mx(v[9], v[41]); v[9] = t; }
    { uint32_t t = op.mn(v[10], v[42]); v[42] = op.mx(v[10], v[42]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[43]); v[43] = op.mx(v[11], v[43]); v[11] = t; }
    { uint32_t t = op.mn(v[12], v[44]); v[44] = op.mx(v[12], v[44]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[45]); v[45] = op.mx(v[13], v[45]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[46]); v[46] = op.mx(v[14], v[46]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[47]); v[47] = op.mx(v[15], v[47]); v[15] = t; }
    { uint32_t t = op.mn(v[16], v[48]); v[48] = op.mx(v[16], v[48]); v[16] = t; }
    { uint32_t t = op.mn(v[0], v[16]); v[16] = op.mx(v[0], v[16]); v[0] = t; }
    { uint32_t t = op.mn(v[1], v[17]); v[17] = op.mx(v[1], v[17]); v[1] = t; }
    { uint32_t t = op.mn(v[2], v[18]); v[18] = op.mx(v[2], v[18]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[19]); v[19] = op.mx(v[3], v[19]); v[3] = t; }
    { uint32_t t = op.mn(v[4], v[20]); v[20] = op.mx(v[4], v[20]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[21]); v[21] = op.mx(v[5], v[21]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[22]); v[22] = op.mx(v[6], v[22]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[23]); v[23] = op.mx(v[7], v[23]); v[7] = t; }
    { uint32_t t = op.mn(v[8], v[24]); v[24] = op.mx(v[8], v[24]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[25]); v[25] = op.mx(v[9], v[25]); v[9] = t; }
    { uint32_t t = op.mn(v[10], v[26]); v[26] = op.mx(v[10], v[26]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[27]); v[27] = op.mx(v[11], v[27]); v[11] = t; }
    { uint32_t t = op.mn(v[12], v[28]); v[28] = op.mx(v[12], v[28]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[29]); v[29] = op.mx(v[13], v[29]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[30]); v[30] = op.mx(v[14], v[30]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[31]); v[31] = op.mx(v[15], v[31]); v[15] = t; }
    { uint32_t t = op.mn(v[32], v[48]); v[48] = op.mx(v[32], v[48]); v[32] = t; }
    { uint32_t t = op.mn(v[16], v[32]); v[32] = op.mx(v[16], v[32]); v[16] = t; }
    { uint32_t t = op.mn(v[17], v[33]); v[33] = op.mx(v[17], v[33]); v[17] = t; }
    { uint32_t t = op.mn(v[18], v[34]); v[34] = op.mx(v[18], v[34]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[35]); v[35] = op.mx(v[19], v[35]); v[19] = t; }
    { uint32_t t = op.mn(v[20], v[36]); v[36] = op.mx(v[20], v[36]); v[20] = t; }
    { uint32_t t = op.mn(v[21], v[37]); v[37] = op.mx(v[21], v[37]); v[21] = t; }
    { uint32_t t = op.mn(v[22], v[38]); v[38] = op.mx(v[22], v[38]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[39]); v[39] = op.mx(v[23], v[39]); v[23] = t; }
    { uint32_t t = op.mn(v[24], v[40]); v[40] = op.mx(v[24], v[40]); v[24] = t; }
    { uint32_t t = op.mn(v[25], v[41]); v[41] = op.mx(v[25], v[41]); v[25] = t; }
    { uint32_t t = op.mn(v[26], v[42]); v[42] = op.mx(v[26], v[42]); v[26] = t; }
    { uint32_t t = op.mn(v[27], v[43]); v[43] = op.mx(v[27], v[43]); v[27] = t; }
    { uint32_t t = op.mn(v[28], v[44]); v[44] = op.mx(v[28], v[44]); v[28] = t; }
    { uint32_t t = op.mn(v[29], v[45]); v[45] = op.mx(v[29], v[45]); v[29] = t; }
    { uint32_t t = op.mn(v[30], v[46]); v[46] = op.mx(v[30], v[46]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[47]); v[47] = op.mx(v[31], v[47]); v[31] = t; }
    { uint32_t t = op.mn(v[0], v[8]); v[8] = op.mx(v[0], v[8]); v[0] = t; }
    { uint32_t t = op.mn(v[1], v[9]); v[9] = op.mx(v[1], v[9]); v[1] = t; }
    { uint32_t t = op.mn(v[2], v[10]); v[10] = op.mx(v[2], v[10]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[11]); v[11] = op.mx(v[3], v[11]); v[3] = t; }
    { uint32_t t = op.mn(v[4], v[12]); v[12] = op.mx(v[4], v[12]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[13]); v[13] = op.mx(v[5], v[13]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[14]); v[14] = op.mx(v[6], v[14]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[15]); v[15] = op.mx(v[7], v[15]); v[7] = t; }
    { uint32_t t = op.mn(v[16], v[24]); v[24] = op.mx(v[16], v[24]); v[16] = t; }
    { uint32_t t = op.mn(v[17], v[25]); v[25] = op.mx(v[17], v[25]); v[17] = t; }
    { uint32_t t = op.mn(v[18], v[26]); v[26] = op.mx(v[18], v[26]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[27]); v[27] = op.mx(v[19], v[27]); v[19] = t; }
    { uint32_t t = op.mn(v[20], v[28]); v[28] = op.mx(v[20], v[28]); v[20] = t; }
    { uint32_t t = op.mn(v[21], v[29]); v[29] = op.mx(v[21], v[29]); v[21] = t; }
    { uint32_t t = op.mn(v[22], v[30]); v[30] = op.mx(v[22], v[30]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[31]); v[31] = op.mx(v[23], v[31]); v[23] = t; }
    { uint32_t t = op.mn(v[32], v[40]); v[40] = op.mx(v[32], v[40]); v[32] = t; }
    { uint32_t t = op.mn(v[33], v[41]); v[41] = op.mx(v[33], v[41]); v[33] = t; }
    { uint32_t t = op.mn(v[34], v[42]); v[42] = op.mx(v[34], v[42]); v[34] = t; }
    { uint32_t t = op.mn(v[35], v[43]); v[43] = op.mx(v[35], v[43]); v[35] = t; }
    { uint32_t t = op.mn(v[36], v[44]); v[44] = op.mx(v[36], v[44]); v[36] = t; }
    { uint32_t t = op.mn(v[37], v[45]); v[45] = op.mx(v[37], v[45]); v[37] = t; }
    { uint32_t t = op.mn(v[38], v[46]); v[46] = op.mx(v[38], v[46]); v[38] = t; }
    { uint32_t t = op.mn(v[39], v[47]); v[47] = op.mx(v[39], v[47]); v[39] = t; }
    { uint32_t t = op.mn(v[8], v[32]); v[32] = op.mx(v[8], v[32]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[33]); v[33] = op.mx(v[9], v[33]); v[9] = t; }
    { uint32_t t = op.mn(v[10], v[34]); v[34] = op.mx(v[10], v[34]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[35]); v[35] = op.mx(v[11], v[35]); v[11] = t; }
    { uint32_t t = op.mn(v[12], v[36]); v[36] = op.mx(v[12], v[36]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[37]); v[37] = op.mx(v[13], v[37]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[38]); v[38] = op.mx(v[14], v[38]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[39]); v[39] = op.mx(v[15], v[39]); v[15] = t; }
    { uint32_t t = op.mn(v[24], v[48]); v[48] = op.mx(v[24], v[48]); v[24] = t; }
    { uint32_t t = op.mn(v[8], v[16]); v[16] = op.mx(v[8], v[16]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[17]); v[17] = op.mx(v[9], v[17]); v[9] = t; }
    { uint32_t t = op.mn(v[10], v[18]); v[18] = op.mx(v[10], v[18]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[19]); v[19] = op.mx(v[11], v[19]); v[11] = t; }
    { uint32_t t = op.mn(v[12], v[20]); v[20] = op.mx(v[12], v[20]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[21]); v[21] = op.mx(v[13], v[21]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[22]); v[22] = op.mx(v[14], v[22]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[23]); v[23] = op.mx(v[15], v[23]); v[15] = t; }
    { uint32_t t = op.mn(v[24], v[32]); v[32] = op.mx(v[24], v[32]); v[24] = t; }
    { uint32_t t = op.mn(v[25], v[33]); v[33] = op.mx(v[25], v[33]); v[25] = t; }
    { uint32_t t = op.mn(v[26], v[34]); v[34] = op.mx(v[26], v[34]); v[26] = t; }
    { uint32_t t = op.mn(v[27], v[35]); v[35] = op.mx(v[27], v[35]); v[27] = t; }
    { uint32_t t = op.mn(v[28], v[36]); v[36] = op.mx(v[28], v[36]); v[28] = t; }
    { uint32_t t = op.mn(v[29], v[37]); v[37] = op.mx(v[29], v[37]); v[29] = t; }
    { uint32_t t = op.mn(v[30], v[38]); v[38] = op.mx(v[30], v[38]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[39]); v[39] = op.mx(v[31], v[39]); v[31] = t; }
    { uint32_t t = op.mn(v[40], v[48]); v[48] = op.mx(v[40], v[48]); v[40] = t; }
    { uint32_t t = op.mn(v[0], v[4]); v[4] = op.mx(v[0], v[4]); v[0] = t; }
    { uint32_t t = op.mn(v[1], v[5]); v[5] = op.mx(v[1], v[5]); v[1] = t; }
    { uint32_t t = op.mn(v[2], v[6]); v[6] = op.mx(v[2], v[6]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[7]); v[7] = op.mx(v[3], v[7]); v[3] = t; }
    { uint32_t t = op.mn(v[8], v[12]); v[12] = op.mx(v[8], v[12]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[13]); v[13] = op.mx(v[9], v[13]); v[9] = t; }
    { uint32_t t = op.mn(v[10], v[14]); v[14] = op.mx(v[10], v[14]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[15]); v[15] = op.mx(v[11], v[15]); v[11] = t; }
    { uint32_t t = op.mn(v[16], v[20]); v[20] = op.mx(v[16], v[20]); v[16] = t; }
    { uint32_t t = op.mn(v[17], v[21]); v[21] = op.mx(v[17], v[21]); v[17] = t; }
    { uint32_t t = op.mn(v[18], v[22]); v[22] = op.mx(v[18], v[22]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[23]); v[23] = op.mx(v[19], v[23]); v[19] = t; }
    { uint32_t t = op.mn(v[24], v[28]); v[28] = op.mx(v[24], v[28]); v[24] = t; }
    { uint32_t t = op.mn(v[25], v[29]); v[29] = op.mx(v[25], v[29]); v[25] = t; }
    { uint32_t t = op.mn(v[26], v[30]); v[30] = op.mx(v[26], v[30]); v[26] = t; }
    { uint32_t t = op.mn(v[27], v[31]); v[31] = op.mx(v[27], v[31]); v[27] = t; }
    { uint32_t t = op.mn(v[32], v[36]); v[36] = op.mx(v[32], v[36]); v[32] = t; }
    { uint32_t t = op.mn(v[33], v[37]); v[37] = op.mx(v[33], v[37]); v[33] = t; }
    { uint32_t t = op.mn(v[34], v[38]); v[38] = op.mx(v[34], v[38]); v[34] = t; }
    { uint32_t t = op.mn(v[35], v[39]); v[39] = op.mx(v[35], v[39]); v[35] = t; }
    { uint32_t t = op.mn(v[40], v[44]); v[44] = op.mx(v[40], v[44]); v[40] = t; }
    { uint32_t t = op.mn(v[41], v[45]); v[45] = op.mx(v[41], v[45]); v[41] = t; }
    { uint32_t t = op.mn(v[42], v[46]); v[46] = op.mx(v[42], v[46]); v[42] = t; }
    { uint32_t t = op.mn(v[43], v[47]); v[47] = op.mx(v[43], v[47]); v[43] = t; }
    { uint32_t t = op.mn(v[4], v[32]); v[32] = op.mx(v[4], v[32]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[33]); v[33] = op.mx(v[5], v[33]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[34]); v[34] = op.mx(v[6], v[34]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[35]); v[35] = op.mx(v[7], v[35]); v[7] = t; }
    { uint32_t t = op.mn(v[12], v[40]); v[40] = op.mx(v[12], v[40]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[41]); v[41] = op.mx(v[13], v[41]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[42]); v[42] = op.mx(v[14], v[42]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[43]); v[43] = op.mx(v[15], v[43]); v[15] = t; }
    { uint32_t t = op.mn(v[20], v[48]); v[48] = op.mx(v[20], v[48]); v[20] = t; }
    { uint32_t t = op.mn(v[4], v[16]); v[16] = op.mx(v[4], v[16]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[17]); v[17] = op.mx(v[5], v[17]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[18]); v[18] = op.mx(v[6], v[18]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[19]); v[19] = op.mx(v[7], v[19]); v[7] = t; }
    { uint32_t t = op.mn(v[12], v[24]); v[24] = op.mx(v[12], v[24]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[25]); v[25] = op.mx(v[13], v[25]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[26]); v[26] = op.mx(v[14], v[26]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[27]); v[27] = op.mx(v[15], v[27]); v[15] = t; }
    { uint32_t t = op.mn(v[20], v[32]); v[32] = op.mx(v[20], v[32]); v[20] = t; }
    { uint32_t t = op.mn(v[21], v[33]); v[33] = op.mx(v[21], v[33]); v[21] = t; }
    { uint32_t t = op.mn(v[22], v[34]); v[34] = op.mx(v[22], v[34]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[35]); v[35] = op.mx(v[23], v[35]); v[23] = t; }
    { uint32_t t = op.mn(v[28], v[40]); v[40] = op.mx(v[28], v[40]); v[28] = t; }
    { uint32_t t = op.mn(v[29], v[41]); v[41] = op.mx(v[29], v[41]); v[29] = t; }
    { uint32_t t = op.mn(v[30], v[42]); v[42] = op.mx(v[30], v[42]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[43]); v[43] = op.mx(v[31], v[43]); v[31] = t; }
    { uint32_t t = op.mn(v[36], v[48]); v[48] = op.mx(v[36], v[48]); v[36] = t; }
    { uint32_t t = op.mn(v[4], v[8]); v[8] = op.mx(v[4], v[8]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[9]); v[9] = op.mx(v[5], v[9]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[10]); v[10] = op.mx(v[6], v[10]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[11]); v[11] = op.mx(v[7], v[11]); v[7] = t; }
    { uint32_t t = op.mn(v[12], v[16]); v[16] = op.mx(v[12], v[16]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[17]); v[17] = op.mx(v[13], v[17]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[18]); v[18] = op.mx(v[14], v[18]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[19]); v[19] = op.mx(v[15], v[19]); v[15] = t; }
    { uint32_t t = op.mn(v[20], v[24]); v[24] = op.mx(v[20], v[24]); v[20] = t; }
    { uint32_t t = op.mn(v[21], v[25]); v[25] = op.mx(v[21], v[25]); v[21] = t; }
    { uint32_t t = op.mn(v[22], v[26]); v[26] = op.mx(v[22], v[26]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[27]); v[27] = op.mx(v[23], v[27]); v[23] = t; }
    { uint32_t t = op.mn(v[28], v[32]); v[32] = op.mx(v[28], v[32]); v[28] = t; }
    { uint32_t t = op.mn(v[29], v[33]); v[33] = op.mx(v[29], v[33]); v[29] = t; }
    { uint32_t t = op.mn(v[30], v[34]); v[34] = op.mx(v[30], v[34]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[35]); v[35] = op.mx(v[31], v[35]); v[31] = t; }
    { uint32_t t = op.mn(v[36], v[40]); v[40] = op.mx(v[36], v[40]); v[36] = t; }
    { uint32_t t = op.mn(v[37], v[41]); v[41] = op.mx(v[37], v[41]); v[37] = t; }
    { uint32_t t = op.mn(v[38], v[42]); v[42] = op.mx(v[38], v[42]); v[38] = t; }
    { uint32_t t = op.mn(v[39], v[43]); v[43] = op.mx(v[39], v[43]); v[39] = t; }
    { uint32_t t = op.mn(v[44], v[48]); v[48] = op.mx(v[44], v[48]); v[44] = t; }
    { uint32_t t = op.mn(v[0], v[2]); v[2] = op.mx(v[0], v[2]); v[0] = t; }
    { uint32_t t = op.mn(v[1], v[3]); v[3] = op.mx(v[1], v[3]); v[1] = t; }
    { uint32_t t = op.mn(v[4], v[6]); v[6] = op.mx(v[4], v[6]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[7]); v[7] = op.mx(v[5], v[7]); v[5] = t; }
    { uint32_t t = op.mn(v[8], v[10]); v[10] = op.mx(v[8], v[10]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[11]); v[11] = op.mx(v[9], v[11]); v[9] = t; }
    { uint32_t t = op.mn(v[12], v[14]); v[14] = op.mx(v[12], v[14]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[15]); v[15] = op.mx(v[13], v[15]); v[13] = t; }
    { uint32_t t = op.mn(v[16], v[18]); v[18] = op.mx(v[16], v[18]); v[16] = t; }
    { uint32_t t = op.mn(v[17], v[19]); v[19] = op.mx(v[17], v[19]); v[17] = t; }
    { uint32_t t = op.mn(v[20], v[22]); v[22] = op.mx(v[20], v[22]); v[20] = t; }
    { uint32_t t = op.mn(v[21], v[23]); v[23] = op.mx(v[21], v[23]); v[21] = t; }
    { uint32_t t = op.mn(v[24], v[26]); v[26] = op.mx(v[24], v[26]); v[24] = t; }
    { uint32_t t = op.mn(v[25], v[27]); v[27] = op.mx(v[25], v[27]); v[25] = t; }
    { uint32_t t = op.mn(v[28], v[30]); v[30] = op.mx(v[28], v[30]); v[28] = t; }
    { uint32_t t = op.mn(v[29], v[31]); v[31] = op.mx(v[29], v[31]); v[29] = t; }
    { uint32_t t = op.mn(v[32], v[34]); v[34] = op.mx(v[32], v[34]); v[32] = t; }
    { uint32_t t = op.mn(v[33], v[35]); v[35] = op.mx(v[33], v[35]); v[33] = t; }
    { uint32_t t = op.mn(v[36], v[38]); v[38] = op.mx(v[36], v[38]); v[36] = t; }
    { uint32_t t = op.mn(v[37], v[39]); v[39] = op.mx(v[37], v[39]); v[37] = t; }
    { uint32_t t = op.mn(v[40], v[42]); v[42] = op.mx(v[40], v[42]); v[40] = t; }
    { uint32_t t = op.mn(v[41], v[43]); v[43] = op.mx(v[41], v[43]); v[41] = t; }
    { uint32_t t = op.mn(v[44], v[46]); v[46] = op.mx(v[44], v[46]); v[44] = t; }
    { uint32_t t = op.mn(v[45], v[47]); v[47] = op.mx(v[45], v[47]); v[45] = t; }
    { uint32_t t = op.mn(v[2], v[32]); v[32] = op.mx(v[2], v[32]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[33]); v[33] = op.mx(v[3], v[33]); v[3] = t; }
    { uint32_t t = op.mn(v[6], v[36]); v[36] = op.mx(v[6], v[36]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[37]); v[37] = op.mx(v[7], v[37]); v[7] = t; }
    { uint32_t t = op.mn(v[10], v[40]); v[40] = op.mx(v[10], v[40]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[41]); v[41] = op.mx(v[11], v[41]); v[11] = t; }
    { uint32_t t = op.mn(v[14], v[44]); v[44] = op.mx(v[14], v[44]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[45]); v[45] = op.mx(v[15], v[45]); v[15] = t; }
    { uint32_t t = op.mn(v[18], v[48]); v[48] = op.mx(v[18], v[48]); v[18] = t; }
    { uint32_t t = op.mn(v[2], v[16]); v[16] = op.mx(v[2], v[16]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[17]); v[17] = op.mx(v[3], v[17]); v[3] = t; }
    { uint32_t t = op.mn(v[6], v[20]); v[20] = op.mx(v[6], v[20]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[21]); v[21] = op.mx(v[7], v[21]); v[7] = t; }
    { uint32_t t = op.mn(v[10], v[24]); v[24] = op.mx(v[10], v[24]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[25]); v[25] = op.mx(v[11], v[25]); v[11] = t; }
    { uint32_t t = op.mn(v[14], v[28]); v[28] = op.mx(v[14], v[28]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[29]); v[29] = op.mx(v[15], v[29]); v[15] = t; }
    { uint32_t t = op.mn(v[18], v[32]); v[32] = op.mx(v[18], v[32]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[33]); v[33] = op.mx(v[19], v[33]); v[19] = t; }
    { uint32_t t = op.mn(v[22], v[36]); v[36] = op.mx(v[22], v[36]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[37]); v[37] = op.mx(v[23], v[37]); v[23] = t; }
    { uint32_t t = op.mn(v[26], v[40]); v[40] = op.mx(v[26], v[40]); v[26] = t; }
    { uint32_t t = op.mn(v[27], v[41]); v[41] = op.mx(v[27], v[41]); v[27] = t; }
    { uint32_t t = op.mn(v[30], v[44]); v[44] = op.mx(v[30], v[44]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[45]); v[45] = op.mx(v[31], v[45]); v[31] = t; }
    { uint32_t t = op.mn(v[34], v[48]); v[48] = op.mx(v[34], v[48]); v[34] = t; }
    { uint32_t t = op.mn(v[2], v[8]); v[8] = op.mx(v[2], v[8]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[9]); v[9] = op.mx(v[3], v[9]); v[3] = t; }
    { uint32_t t = op.mn(v[6], v[12]); v[12] = op.mx(v[6], v[12]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[13]); v[13] = op.mx(v[7], v[13]); v[7] = t; }
    { uint32_t t = op.mn(v[10], v[16]); v[16] = op.mx(v[10], v[16]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[17]); v[17] = op.mx(v[11], v[17]); v[11] = t; }
    { uint32_t t = op.mn(v[14], v[20]); v[20] = op.mx(v[14], v[20]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[21]); v[21] = op.mx(v[15], v[21]); v[15] = t; }
    { uint32_t t = op.mn(v[18], v[24]); v[24] = op.mx(v[18], v[24]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[25]); v[25] = op.mx(v[19], v[25]); v[19] = t; }
    { uint32_t t = op.mn(v[22], v[28]); v[28] = op.mx(v[22], v[28]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[29]); v[29] = op.mx(v[23], v[29]); v[23] = t; }
    { uint32_t t = op.mn(v[26], v[32]); v[32] = op.mx(v[26], v[32]); v[26] = t; }
    { uint32_t t = op.mn(v[27], v[33]); v[33] = op.mx(v[27], v[33]); v[27] = t; }
    { uint32_t t = op.mn(v[30], v[36]); v[36] = op.mx(v[30], v[36]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[37]); v[37] = op.mx(v[31], v[37]); v[31] = t; }
    { uint32_t t = op.mn(v[34], v[40]); v[40] = op.mx(v[34], v[40]); v[34] = t; }
    { uint32_t t = op.mn(v[35], v[41]); v[41] = op.mx(v[35], v[41]); v[35] = t; }
    { uint32_t t = op.mn(v[38], v[44]); v[44] = op.mx(v[38], v[44]); v[38] = t; }
    { uint32_t t = op.mn(v[39], v[45]); v[45] = op.mx(v[39], v[45]); v[39] = t; }
    { uint32_t t = op.mn(v[42], v[48]); v[48] = op.mx(v[42], v[48]); v[42] = t; }
    { uint32_t t = op.mn(v[2], v[4]); v[4] = op.mx(v[2], v[4]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[5]); v[5] = op.mx(v[3], v[5]); v[3] = t; }
    { uint32_t t = op.mn(v[6], v[8]); v[8] = op.mx(v[6], v[8]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[9]); v[9] = op.mx(v[7], v[9]); v[7] = t; }
    { uint32_t t = op.mn(v[10], v[12]); v[12] = op.mx(v[10], v[12]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[13]); v[13] = op.mx(v[11], v[13]); v[11] = t; }
    { uint32_t t = op.mn(v[14], v[16]); v[16] = op.mx(v[14], v[16]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[17]); v[17] = op.mx(v[15], v[17]); v[15] = t; }
    { uint32_t t = op.mn(v[18], v[20]); v[20] = op.mx(v[18], v[20]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[21]); v[21] = op.mx(v[19], v[21]); v[19] = t; }
    { uint32_t t = op.mn(v[22], v[24]); v[24] = op.mx(v[22], v[24]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[25]); v[25] = op.mx(v[23], v[25]); v[23] = t; }
    { uint32_t t = op.mn(v[26], v[28]); v[28] = op.mx(v[26], v[28]); v[26] = t; }
    { uint32_t t = op.mn(v[27], v[29]); v[29] = op.mx(v[27], v[29]); v[27] = t; }
    { uint32_t t = op.mn(v[30], v[32]); v[32] = op.mx(v[30], v[32]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[33]); v[33] = op.mx(v[31], v[33]); v[31] = t; }
    { uint32_t t = op.mn(v[34], v[36]); v[36] = op.mx(v[34], v[36]); v[34] = t; }
    { uint32_t t = op.mn(v[35], v[37]); v[37] = op.mx(v[35], v[37]); v[35] = t; }
    { uint32_t t = op.mn(v[38], v[40]); v[40] = op.mx(v[38], v[40]); v[38] = t; }
    { uint32_t t = op.mn(v[39], v[41]); v[41] = op.mx(v[39], v[41]); v[39] = t; }
    { uint32_t t = op.mn(v[42], v[44]); v[44] = op.mx(v[42], v[44]); v[42] = t; }
    { uint32_t t = op.mn(v[43], v[45]); v[45] = op.mx(v[43], v[45]); v[43] = t; }
    { uint32_t t = op.mn(v[46], v[48]); v[48] = op.mx(v[46], v[48]); v[46] = t; }
    v[1] = op.mx(v[0], v[1]);
    v[3] = op.mx(v[2], v[3]);
    v[5] = op.mx(v[4], v[5]);
    v[7] = op.mx(v[6], v[7]);
    v[9] = op.mx(v[8], v[9]);
    v[11] = op.mx(v[10], v[11]);
    v[13] = op.mx(v[12], v[13]);
    v[15] = op.mx(v[14], v[15]);
    v[17] = op.mx(v[16], v[17]);
    v[19] = op.mx(v[18], v[19]);
    v[21] = op.mx(v[20], v[21]);
    v[23] = op.mx(v[22], v[23]);
    v[24] = op.mn(v[24], v[25]);
    v[26] = op.mn(v[26], v[27]);
    v[28] = op.mn(v[28], v[29]);
    v[30] = op.mn(v[30], v[31]);
    v[32] = op.mn(v[32], v[33]);
    v[34] = op.mn(v[34], v[35]);
    v[36] = op.mn(v[36], v[37]);
    v[38] = op.mn(v[38], v[39]);
    v[40] = op.mn(v[40], v[41]);
    v[42] = op.mn(v[42], v[43]);
    v[44] = op.mn(v[44], v[45]);
    v[46] = op.mn(v[46], v[47]);
    v[32] = op.mx(v[1], v[32]);
    v[34] = op.mx(v[3], v[34]);
    v[36] = op.mx(v[5], v[36]);
    v[38] = op.mx(v[7], v[38]);
    v[9] = op.mn(v[9], v[40]);
    v[11] = op.mn(v[11], v[42]);
    v[13] = op.mn(v[13], v[44]);
    v[15] = op.mn(v[15], v[46]);
    v[17] = op.mn(v[17], v[48]);
    v[24] = op.mx(v[9], v[24]);
    v[26] = op.mx(v[11], v[26]);
    v[28] = op.mx(v[13], v[28]);
    v[30] = op.mx(v[15], v[30]);
    v[17] = op.mn(v[17], v[32]);
    v[19] = op.mn(v[19], v[34]);
    v[21] = op.mn(v[21], v[36]);
    v[23] = op.mn(v[23], v[38]);
    v[24] = op.mx(v[17], v[24]);
    v[26] = op.mx(v[19], v[26]);
    v[21] = op.mn(v[21], v[28]);
    v[23] = op.mn(v[23], v[30]);
    v[24] = op.mx(v[21], v[24]);
    v[23] = op.mn(v[23], v[26]);
    v[24] = op.mx(v[23], v[24]);
    return v[24];
  }
};

// k=9: 661 compare-exchanges, 1242 min/max ops
template <> struct MedianNet<9> {
  static constexpr int kOps = 1242;
  template <class Op> __device__ __forceinline__ static uint32_t run(uint32_t (&v)[81], Op op) {
    { uint32_t t = op.mn(v[0], v[64]); v[64] = op.mx(v[0], v[64]); v[0] = t; }
    { uint32_t t = op.mn(v[1], v[65]); v[65] = op.mx(v[1], v[65]); v[1] = t; }
    { uint32_t t = op.mn(v[2], v[66]); v[66] = op.mx(v[2], v[66]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[67]); v[67] = op.mx(v[3], v[67]); v[3] = t; }
    { uint32_t t = op.mn(v[4], v[68]); v[68] = op.mx(v[4], v[68]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[69]); v[69] = op.mx(v[5], v[69]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[70]); v[70] = op.mx(v[6], v[70]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[71]); v[71] = op.mx(v[7], v[71]); v[7] = t; }
    { uint32_t t = op.mn(v[8], v[72]); v[72] = op.mx(v[8], v[72]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[73]); v[73] = op.mx(v[9], v[73]); v[9] = t; }
    { uint32_t t = op.mn(v[10], v[74]); v[74] = op.mx(v[10], v[74]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[75]); v[75] = op.mx(v[11], v[75]); v[11] = t; }
    { uint32_t t = op.mn(v[12], v[76]); v[76] = op.mx(v[12], v[76]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[77]); v[77] = op.mx(v[13], v[77]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[78]); v[78] = op.mx(v[14], v[78]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[79]); v[79] = op.mx(v[15], v[79]); v[15] = t; }
    { uint32_t t = op.mn(v[16], v[80]); v[80] = op.mx(v[16], v[80]); v[16] = t; }
    { uint32_t t = op.mn(v[0], v[32]); v[32] = op.mx(v[0], v[32]); v[0] = t; }
    { uint32_t t = op.mn(v[1], v[33]); v[33] = op.mx(v[1], v[33]); v[1] = t; }
    { uint32_t t = op.mn(v[2], v[34]); v[34] = op.mx(v[2], v[34]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[35]); v[35] = op.mx(v[3], v[35]); v[3] = t; }
    { uint32_t t = op.mn(v[4], v[36]); v[36] = op.mx(v[4], v[36]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[37]); v[37] = op.mx(v[5], v[37]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[38]); v[38] = op.mx(v[6], v[38]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[39]); v[39] = op.mx(v[7], v[39]); v[7] = t; }
    { uint32_t t = op.mn(v[8], v[40]); v[40] = op.mx(v[8], v[40]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[41]); v[41] = op.mx(v[9], v[41]); v[9] = t; }
    { uint32_t t = op.mn(v[10], v[42]); v[42] = op.mx(v[10], v[42]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[43]); v[43] = op.mx(v[11], v[43]); v[11] = t; }
    { uint32_t t = op.mn(v[12], v[44]); v[44] = op.mx(v[12], v[44]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[45]); v[45] = op.mx(v[13], v[45]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[46]); v[46] = op.mx(v[14], v[46]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[47]); v[47] = op.mx(v[15], v[47]); v[15] = t; }
    { uint32_t t = op.mn(v[16], v[48]); v[48] = op.mx(v[16], v[48]); v[16] = t; }
    { uint32_t t = op.mn(v[17], v[49]); v[49] = op.mx(v[17], v[49]); v[17] = t; }
    { uint32_t t = op.mn(v[18], v[50]); v[50] = op.mx(v[18], v[50]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[51]); v[51] = op.mx(v[19], v[51]); v[19] = t; }
    { uint32_t t = op.mn(v[20], v[52]); v[52] = op.mx(v[20], v[52]); v[20] = t; }
    { uint32_t t = op.mn(v[21], v[53]); v[53] = op.mx(v[21], v[53]); v[21] = t; }
    { uint32_t t = op.mn(v[22], v[54]); v[54] = op.mx(v[22], v[54]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[55]); v[55] = op.mx(v[23], v[55]); v[23] = t; }
    { uint32_t t = op.mn(v[24], v[56]); v[56] = op.mx(v[24], v[56]); v[24] = t; }
    { uint32_t t = op.mn(v[25], v[57]); v[57] = op.mx(v[25], v[57]); v[25] = t; }
    { uint32_t t = op.mn(v[26], v[58]); v[58] = op.mx(v[26], v[58]); v[26] = t; }
    { uint32_t t = op.mn(v[27], v[59]); v[59] = op.mx(v[27], v[59]); v[27] = t; }
    { uint32_t t = op.mn(v[28], v[60]); v[60] = op.mx(v[28], v[60]); v[28] = t; }
    { uint32_t t = op.mn(v[29], v[61]); v[61] = op.mx(v[29], v[61]); v[29] = t; }
    { uint32_t t = op.mn(v[30], v[62]); v[62] = op.mx(v[30], v[62]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[63]); v[63] = op.mx(v[31], v[63]); v[31] = t; }
    { uint32_t t = op.mn(v[32], v[64]); v[64] = op.mx(v[32], v[64]); v[32] = t; }
    { uint32_t t = op.mn(v[33], v[65]); v[65] = op.mx(v[33], v[65]); v[33] = t; }
    { uint32_t t = op.mn(v[34], v[66]); v[66] = op.mx(v[34], v[66]); v[34] = t; }
    { uint32_t t = op.mn(v[35], v[67]); v[67] = op.mx(v[35], v[67]); v[35] = t; }
    { uint32_t t = op.mn(v[36], v[68]); v[68] = op.mx(v[36], v[68]); v[36] = t; }
    { uint32_t t = op.mn(v[37], v[69]); v[69] = op.mx(v[37], v[69]); v[37] = t; }
    { uint32_t t = op.mn(v[38], v[70]); v[70] = op.mx(v[38], v[70]); v[38] = t; }
    { uint32_t t = op.mn(v[39], v[71]); v[71] = op.mx(v[39], v[71]); v[39] = t; }
    { uint32_t t = op.mn(v[40], v[72]); v[72] = op.mx(v[40], v[72]); v[40] = t; }
    { uint32_t t = op.mn(v[41], v[73]); v[73] = op.mx(v[41], v[73]); v[41] = t; }
    { uint32_t t = op.mn(v[42], v[74]); v[74] = op.mx(v[42], v[74]); v[42] = t; }
    { uint32_t t = op.mn(v[43], v[75]); v[75] = op.mx(v[43], v[75]); v[43] = t; }
    { uint32_t t = op.mn(v[44], v[76]); v[76] = op.mx(v[44], v[76]); v[44] = t; }
    { uint32_t t = op.mn(v[45], v[77]); v[77] = op.mx(v[45], v[77]); v[45] = t; }
    { uint32_t t = op.mn(v[46], v[78]); v[78] = op.mx(v[46], v[78]); v[46] = t; }
    { uint32_t t = op.mn(v[47], v[79]); v[79] = op.mx(v[47], v[79]); v[47] = t; }
    { uint32_t t = op.mn(v[48], v[80]); v[80] = op.mx(v[48], v[80]); v[48] = t; }
    { uint32_t t = op.mn(v[0], v[16]); v[16] = op.mx(v[0], v[16]); v[0] = t; }
    { uint32_t t = op.mn(v[1], v[17]); v[17] = op.mx(v[1], v[17]); v[1] = t; }
    { uint32_t t = op.mn(v[2], v[18]); v[18] = op.mx(v[2], v[18]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[19]); v[19] = op.mx(v[3], v[19]); v[3] = t; }
    { uint32_t t = op.mn(v[4], v[20]); v[20] = op.mx(v[4], v[20]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[21]); v[21] = op.mx(v[5], v[21]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[22]); v[22] = op.mx(v[6], v[22]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[23]); v[23] = op.mx(v[7], v[23]); v[7] = t; }
    { uint32_t t = op.mn(v[8], v[24]); v[24] = op.mx(v[8], v[24]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[25]); v[25] = op.mx(v[9], v[25]); v[9] = t; }
    { uint32_t t = op.mn(v[10], v[26]); v[26] = op.mx(v[10], v[26]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[27]); v[27] = op.mx(v[11], v[27]); v[11] = t; }
    { uint32_t t = op.mn(v[12], v[28]); v[28] = op.mx(v[12], v[28]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[29]); v[29] = op.mx(v[13], v[29]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[30]); v[30] = op.mx(v[14], v[30]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[31]); v[31] = op.mx(v[15], v[31]); v[15] = t; }
    { uint32_t t = op.mn(v[32], v[48]); v[48] = op.mx(v[32], v[48]); v[32] = t; }
    { uint32_t t = op.mn(v[33], v[49]); v[49] = op.mx(v[33], v[49]); v[33] = t; }
    { uint32_t t = op.mn(v[34], v[50]); v[50] = op.mx(v[34], v[50]); v[34] = t; }
    { uint32_t t = op.mn(v[35], v[51]); v[51] = op.mx(v[35], v[51]); v[35] = t; }
    { uint32_t t = op.mn(v[36], v[52]); v[52] = op.mx(v[36], v[52]); v[36] = t; }
    { uint32_t t = op.mn(v[37], v[53]); v[53] = op.mx(v[37], v[53]); v[37] = t; }
    { uint32_t t = op.mn(v[38], v[54]); v[54] = op.mx(v[38], v[54]); v[38] = t; }
    { uint32_t t = op.mn(v[39], v[55]); v[55] = op.mx(v[39], v[55]); v[39] = t; }
    { uint32_t t = op.mn(v[40], v[56]); v[56] = op.mx(v[40], v[56]); v[40] = t; }
    { uint32_t t = op.mn(v[41], v[57]); v[57] = op.mx(v[41], v[57]); v[41] = t; }
    { uint32_t t = op.mn(v[42], v[58]); v[58] = op.mx(v[42], v[58]); v[42] = t; }
    { uint32_t t = op.mn(v[43], v[59]); v[59] = op.mx(v[43], v[59]); v[43] = t; }
    { uint32_t t = op.mn(v[44], v[60]); v[60] = op.mx(v[44], v[60]); v[44] = t; }
    { uint32_t t = op.mn(v[45], v[61]); v[61] = op.mx(v[45], v[61]); v[45] = t; }
    { uint32_t t = op.mn(v[46], v[62]); v[62] = op.mx(v[46], v[62]); v[46] = t; }
    { uint32_t t = op.mn(v[47], v[63]); v[63] = op.mx(v[47], v[63]); v[47] = t; }
    { uint32_t t = op.mn(v[64], v[80]); v[80] = op.mx(v[64], v[80]); v[64] = t; }
    { uint32_t t = op.mn(v[16], v[64]); v[64] = op.mx(v[16], v[64]); v[16] = t; }
    { uint32_t t = op.mn(v[17], v[65]); v[65] = op.mx(v[17], v[65]); v[17] = t; }
    { uint32_t t = op.mn(v[18], v[66]); v[66] = op.mx(v[18], v[66]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[67]); v[67] = op.mx(v[19], v[67]); v[19] = t; }
    { uint32_t t = op.mn(v[20], v[68]); v[68] = op.mx(v[20], v[68]); v[20] = t; }
    { uint32_t t = op.mn(v[21], v[69]); v[69] = op.mx(v[21], v[69]); v[21] = t; }
    { uint32_t t = op.mn(v[22], v[70]); v[70] = op.mx(v[22], v[70]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[71]); v[71] = op.mx(v[23], v[71]); v[23] = t; }
    { uint32_t t = op.mn(v[24], v[72]); v[72] = op.mx(v[24], v[72]); v[24] = t; }
    { uint32_t t = op.mn(v[25], v[73]); v[73] = op.mx(v[25], v[73]); v[25] = t; }
    { uint32_t t = op.mn(v[26], v[74]); v[74] = op.mx(v[26], v[74]); v[26] = t; }
    { uint32_t t = op.mn(v[27], v[75]); v[75] = op.mx(v[27], v[75]); v[27] = t; }
    { uint32_t t = op.mn(v[28], v[76]); v[76] = op.mx(v[28], v[76]); v[28] = t; }
    { uint32_t t = op.mn(v[29], v[77]); v[77] = op.mx(v[29], v[77]); v[29] = t; }
    { uint32_t t = op.mn(v[30], v[78]); v[78] = op.mx(v[30], v[78]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[79]); v[79] = op.mx(v[31], v[79]); v[31] = t; }
    { uint32_t t = op.mn(v[16], v[32]); v[32] = op.mx(v[16], v[32]); v[16] = t; }
    { uint32_t t = op.mn(v[17], v[33]); v[33] = op.mx(v[17], v[33]); v[17] = t; }
    { uint32_t t = op.mn(v[18], v[34]); v[34] = op.mx(v[18], v[34]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[35]); v[35] = op.mx(v[19], v[35]); v[19] = t; }
    { uint32_t t = op.mn(v[20], v[36]); v[36] = op.mx(v[20], v[36]); v[20] = t; }
    { uint32_t t = op.mn(v[21], v[37]); v[37] = op.mx(v[21], v[37]); v[21] = t; }
    { uint32_t t = op.mn(v[22], v[38]); v[38] = op.mx(v[22], v[38]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[39]); v[39] = op.mx(v[23], v[39]); v[23] = t; }
    { uint32_t t = op.mn(v[24], v[40]); v[40] = op.mx(v[24], v[40]); v[24] = t; }
    { uint32_t t = op.mn(v[25], v[41]); v[41] = op.mx(v[25], v[41]); v[25] = t; }
    { uint32_t t = op.mn(v[26], v[42]); v[42] = op.mx(v[26], v[42]); v[26] = t; }
    { uint32_t t = op.mn(v[27], v[43]); v[43] = op.mx(v[27], v[43]); v[27] = t; }
    { uint32_t t = op.mn(v[28], v[44]); v[44] = op.mx(v[28], v[44]); v[28] = t; }
    { uint32_t t = op.mn(v[29], v[45]); v[45] = op.mx(v[29], v[45]); v[29] = t; }
    { uint32_t t = op.mn(v[30], v[46]); v[46] = op.mx(v[30], v[46]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[47]); v[47] = op.mx(v[31], v[47]); v[31] = t; }
    { uint32_t t = op.mn(v[48], v[64]); v[64] = op.mx(v[48], v[64]); v[48] = t; }
    { uint32_t t = op.mn(v[49], v[65]); v[65] = op.mx(v[49], v[65]); v[49] = t; }
    { uint32_t t = op.mn(v[50], v[66]); v[66] = op.mx(v[50], v[66]); v[50] = t; }
    { uint32_t t = op.mn(v[51], v[67]); v[67] = op.mx(v[51], v[67]); v[51] = t; }
    { uint32_t t = op.mn(v[52], v[68]); v[68] = op.mx(v[52], v[68]); v[52] = t; }
    { uint32_t t = op.mn(v[53], v[69]); v[69] = op.mx(v[53], v[69]); v[53] = t; }
    { uint32_t t = op.mn(v[54], v[70]); v[70] = op.mx(v[54], v[70]); v[54] = t; }
    { uint32_t t = op.mn(v[55], v[71]); v[71] = op.mx(v[55], v[71]); v[55] = t; }
    { uint32_t t = op.mn(v[56], v[72]); v[72] = op.mx(v[56], v[72]); v[56] = t; }
    { uint32_t t = op.mn(v[57], v[73]); v[73] = op.mx(v[57], v[73]); v[57] = t; }
    { uint32_t t = op.mn(v[58], v[74]); v[74] = op.mx(v[58], v[74]); v[58] = t; }
    { uint32_t t = op.mn(v[59], v[75]); v[75] = op.mx(v[59], v[75]); v[59] = t; }
    { uint32_t t = op.mn(v[60], v[76]); v[76] = op.mx(v[60], v[76]); v[60] = t; }
    { uint32_t t = op.mn(v[61], v[77]); v[77] = op.mx(v[61], v[77]); v[61] = t; }
    { uint32_t t = op.mn(v[62], v[78]); v[78] = op.mx(v[62], v[78]); v[62] = t; }
    { uint32_t t = op.mn(v[63], v[79]); v[79] = op.mx(v[63], v[79]); v[63] = t; }
    { uint32_t t = op.mn(v[0], v[8]); v[8] = op.mx(v[0], v[8]); v[0] = t; }
    { uint32_t t = op.mn(v[1], v[9]); v[9] = op.mx(v[1], v[9]); v[1] = t; }
    { uint32_t t = op.mn(v[2], v[10]); v[10] = op.mx(v[2], v[10]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[11]); v[11] = op.mx(v[3], v[11]); v[3] = t; }
    { uint32_t t = op.mn(v[4], v[12]); v[12] = op.mx(v[4], v[12]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[13]); v[13] = op.mx(v[5], v[13]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[14]); v[14] = op.mx(v[6], v[14]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[15]); v[15] = op.mx(v[7], v[15]); v[7] = t; }
    { uint32_t t = op.mn(v[16], v[24]); v[24] = op.mx(v[16], v[24]); v[16] = t; }
    { uint32_t t = op.mn(v[17], v[25]); v[25] = op.mx(v[17], v[25]); v[17] = t; }
    { uint32_t t = op.mn(v[18], v[26]); v[26] = op.mx(v[18], v[26]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[27]); v[27] = op.mx(v[19], v[27]); v[19] = t; }
    { uint32_t t = op.mn(v[20], v[28]); v[28] = op.mx(v[20], v[28]); v[20] = t; }
    { uint32_t t = op.mn(v[21], v[29]); v[29] = op.mx(v[21], v[29]); v[21] = t; }
    { uint32_t t = op.mn(v[22], v[30]); v[30] = op.mx(v[22], v[30]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[31]); v[31] = op.mx(v[23], v[31]); v[23] = t; }
    { uint32_t t = op.mn(v[32], v[40]); v[40] = op.mx(v[32], v[40]); v[32] = t; }
    { uint32_t t = op.mn(v[33], v[41]); v[41] = op.mx(v[33], v[41]); v[33] = t; }
    { uint32_t t = op.mn(v[34], v[42]); v[42] = op.mx(v[34], v[42]); v[34] = t; }
    { uint32_t t = op.mn(v[35], v[43]); v[43] = op.mx(v[35], v[43]); v[35] = t; }
    { uint32_t t = op.mn(v[36], v[44]); v[44] = op.mx(v[36], v[44]); v[36] = t; }
    { uint32_t t = op.mn(v[37], v[45]); v[45] = op.mx(v[37], v[45]); v[37] = t; }
    { uint32_t t = op.mn(v[38], v[46]); v[46] = op.mx(v[38], v[46]); v[38] = t; }
    { uint32_t t = op.mn(v[39], v[47]); v[47] = op.mx(v[39], v[47]); v[39] = t; }
    { uint32_t t = op.mn(v[48], v[56]); v[56] = op.mx(v[48], v[56]); v[48] = t; }
    { uint32_t t = op.mn(v[49], v[57]); v[57] = op.mx(v[49], v[57]); v[49] = t; }
    { uint32_t t = op.mn(v[50], v[58]); v[58] = op.mx(v[50], v[58]); v[50] = t; }
    { uint32_t t = op.mn(v[51], v[59]); v[59] = op.mx(v[51], v[59]); v[51] = t; }
    { uint32_t t = op.mn(v[52], v[60]); v[60] = op.mx(v[52], v[60]); v[52] = t; }
    { uint32_t t = op.mn(v[53], v[61]); v[61] = op.mx(v[53], v[61]); v[53] = t; }
    { uint32_t t = op.mn(v[54], v[62]); v[62] = op.mx(v[54], v[62]); v[54] = t; }
    { uint32_t t = op.mn(v[55], v[63]); v[63] = op.mx(v[55], v[63]); v[55] = t; }
    { uint32_t t = op.mn(v[64], v[72]); v[72] = op.mx(v[64], v[72]); v[64] = t; }
    { uint32_t t = op.mn(v[65], v[73]); v[73] = op.mx(v[65], v[73]); v[65] = t; }
    { uint32_t t = op.mn(v[66], v[74]); v[74] = op.mx(v[66], v[74]); v[66] = t; }
    { uint32_t t = op.mn(v[67], v[75]); v[75] = op.mx(v[67], v[75]); v[67] = t; }
    { uint32_t t = op.mn(v[68], v[76]); v[76] = op.mx(v[68], v[76]); v[68] = t; }
    { uint32_t t = op.mn(v[69], v[77]); v[77] = op.mx(v[69], v[77]); v[69] = t; }
    { uint32_t t = op.mn(v[70], v[78]); v[78] = op.mx(v[70], v[78]); v[70] = t; }
    { uint32_t t = op.mn(v[71], v[79]); v[79] = op.mx(v[71], v[79]); v[71] = t; }
    { uint32_t t = op.mn(v[8], v[64]); v[64] = op.mx(v[8], v[64]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[65]); v[65] = op.mx(v[9], v[65]); v[9] = t; }
    { uint32_t t = op.mn(v[10], v[66]); v[66] = op.mx(v[10], v[66]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[67]); v[67] = op.mx(v[11], v[67]); v[11] = t; }
    { uint32_t t = op.mn(v[12], v[68]); v[68] = op.mx(v[12], v[68]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[69]); v[69] = op.mx(v[13], v[69]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[70]); v[70] = op.mx(v[14], v[70]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[71]); v[71] = op.mx(v[15], v[71]); v[15] = t; }
    { uint32_t t = op.mn(v[24], v[80]); v[80] = op.mx(v[24], v[80]); v[24] = t; }
    { uint32_t t = op.mn(v[8], v[32]); v[32] = op.mx(v[8], v[32]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[33]); v[33] = op.mx(v[9], v[33]); v[9] = t; }
    { uint32_t t = op.mn(v[10], v[34]); v[34] = op.mx(v[10], v[34]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[35]); v[35] = op.mx(v[11], v[35]); v[11] = t; }
    { uint32_t t = op.mn(v[12], v[36]); v[36] = op.mx(v[12], v[36]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[37]); v[37] = op.mx(v[13], v[37]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[38]); v[38] = op.mx(v[14], v[38]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[39]); v[39] = op.mx(v[15], v[39]); v[15] = t; }
    { uint32_t t = op.mn(v[24], v[48]); v[48] = op.mx(v[24], v[48]); v[24] = t; }
    { uint32_t t = op.mn(v[25], v[49]); v[49] = op.mx(v[25], v[49]); v[25] = t; }
    { uint32_t t = op.mn(v[26], v[50]); v[50] = op.mx(v[26], v[50]); v[26] = t; }
    { uint32_t t = op.mn(v[27], v[51]); v[51] = op.mx(v[27], v[51]); v[27] = t; }
    { uint32_t t = op.mn(v[28], v[52]); v[52] = op.mx(v[28], v[52]); v[28] = t; }
    { uint32_t t = op.mn(v[29], v[53]); v[53] = op.mx(v[29], v[53]); v[29] = t; }
    { uint32_t t = op.mn(v[30], v[54]); v[54] = op.mx(v[30], v[54]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[55]); v[55] = op.mx(v[31], v[55]); v[31] = t; }
    { uint32_t t = op.mn(v[40], v[64]); v[64] = op.mx(v[40], v[64]); v[40] = t; }
    { uint32_t t = op.mn(v[41], v[65]); v[65] = op.mx(v[41], v[65]); v[41] = t; }
    { uint32_t t = op.mn(v[42], v[66]); v[66] = op.mx(v[42], v[66]); v[42] = t; }
    { uint32_t t = op.mn(v[43], v[67]); v[67] = op.mx(v[43], v[67]); v[43] = t; }
    { uint32_t t = op.mn(v[44], v[68]); v[68] = op.mx(v[44], v[68]); v[44] = t; }
    { uint32_t t = op.mn(v[45], v[69]); v[69] = op.mx(v[45], v[69]); v[45] = t; }
    { uint32_t t = op.mn(v[46], v[70]); v[70] = op.mx(v[46], v[70]); v[46] = t; }
    { uint32_t t = op.mn(v[47], v[71]); v[71] = op.mx(v[47], v[71]); v[47] = t; }
    { uint32_t t = op.mn(v[56], v[80]); v[80] = op.mx(v[56], v[80]); v[56] = t; }
    { uint32_t t = op.mn(v[8], v[16]); v[16] = op.mx(v[8], v[16]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[17]); v[17] = op.mx(v[9], v[17]); v[9] = t; }
    { uint32_t t = op.mn(v[10], v[18]); v[18] = op.mx(v[10], v[18]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[19]); v[19] = op.mx(v[11], v[19]); v[11] = t; }
    { uint32_t t = op.mn(v[12], v[20]); v[20] = op.mx(v[12], v[20]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[21]); v[21] = op.mx(v[13], v[21]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[22]); v[22] = op.mx(v[14], v[22]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[23]); v[23] = op.mx(v[15], v[23]); v[15] = t; }
    { uint32_t t = op.mn(v[24], v[32]); v[32] = op.mx(v[24], v[32]); v[24] = t; }
    { uint32_t t = op.mn(v[25], v[33]); v[33] = op.mx(v[25], v[33]); v[25] = t; }
    { uint32_t t = op.mn(v[26], v[34]); v[34] = op.mx(v[26], v[34]); v[26] = t; }
    { uint32_t t = op.mn(v[27], v[35]); v[35] = op.mx(v[27], v[35]); v[27] = t; }
    { uint32_t t = op.mn(v[28], v[36]); v[36] = op.mx(v[28], v[36]); v[28] = t; }
    { uint32_t t = op.mn(v[29], v[37]); v[37] = op.mx(v[29], v[37]); v[29] = t; }
    { uint32_t t = op.mn(v[30], v[38]); v[38] = op.mx(v[30], v[38]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[39]); v[39] = op.mx(v[31], v[39]); v[31] = t; }
    { uint32_t t = op.mn(v[40], v[48]); v[48] = op.mx(v[40], v[48]); v[40] = t; }
    { uint32_t t = op.mn(v[41], v[49]); v[49] = op.mx(v[41], v[49]); v[41] = t; }
    { uint32_t t = op.mn(v[42], v[50]); v[50] = op.mx(v[42], v[50]); v[42] = t; }
    { uint32_t t = op.mn(v[43], v[51]); v[51] = op.mx(v[43], v[51]); v[43] = t; }
    { uint32_t t = op.mn(v[44], v[52]); v[52] = op.mx(v[44], v[52]); v[44] = t; }
    { uint32_t t = op.mn(v[45], v[53]); v[53] = op.mx(v[45], v[53]); v[45] = t; }
    { uint32_t t = op.mn(v[46], v[54]); v[54] = op.mx(v[46], v[54]); v[46] = t; }
    { uint32_t t = op.mn(v[47], v[55]); v[55] = op.mx(v[47], v[55]); v[47] = t; }
    { uint32_t t = op.mn(v[56], v[64]); v[64] = op.mx(v[56], v[64]); v[56] = t; }
    { uint32_t t = op.mn(v[57], v[65]); v[65] = op.mx(v[57], v[65]); v[57] = t; }
    { uint32_t t = op.mn(v[58], v[66]); v[66] = op.mx(v[58], v[66]); v[58] = t; }
    { uint32_t t = op.mn(v[59], v[67]); v[67] = op.mx(v[59], v[67]); v[59] = t; }
    { uint32_t t = op.mn(v[60], v[68]); v[68] = op.mx(v[60], v[68]); v[60] = t; }
    { uint32_t t = op.mn(v[61], v[69]); v[69] = op.mx(v[61], v[69]); v[61] = t; }
    { uint32_t t = op.mn(v[62], v[70]); v[70] = op.mx(v[62], v[70]); v[62] = t; }
    { uint32_t t = op.mn(v[63], v[71]); v[71] = op.mx(v[63], v[71]); v[63] = t; }
    { uint32_t t = op.mn(v[72], v[80]); v[80] = op.mx(v[72], v[80]); v[72] = t; }
    { uint32_t t = op.mn(v[0], v[4]); v[4] = op.mx(v[0], v[4]); v[0] = t; }
    { uint32_t t = op.mn(v[1], v[5]); v[5] = op.mx(v[1], v[5]); v[1] = t; }
    { uint32_t t = op.mn(v[2], v[6]); v[6] = op.mx(v[2], v[6]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[7]); v[7] = op.mx(v[3], v[7]); v[3] = t; }
    { uint32_t t = op.mn(v[8], v[12]); v[12] = op.mx(v[8], v[12]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[13]); v[13] = op.mx(v[9], v[13]); v[9] = t; }
    { uint32_t t = op.mn(v[10], v[14]); v[14] = op.mx(v[10], v[14]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[15]); v[15] = op.mx(v[11], v[15]); v[11] = t; }
    { uint32_t t = op.mn(v[16], v[20]); v[20] = op.mx(v[16], v[20]); v[16] = t; }
    { uint32_t t = op.mn(v[17], v[21]); v[21] = op.mx(v[17], v[21]); v[17] = t; }
    { uint32_t t = op.mn(v[18], v[22]); v[22] = op.mx(v[18], v[22]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[23]); v[23] = op.mx(v[19], v[23]); v[19] = t; }
    { uint32_t t = op.mn(v[24], v[28]); v[28] = op.mx(v[24], v[28]); v[24] = t; }
    { uint32_t t = op.mn(v[25], v[29]); v[29] = op.mx(v[25], v[29]); v[25] = t; }
    { uint32_t t = op.mn(v[26], v[30]); v[30] = op.mx(v[26], v[30]); v[26] = t; }
    { uint32_t t = op.mn(v[27], v[31]); v[31] = op.mx(v[27], v[31]); v[27] = t; }
    { uint32_t t = op.mn(v[32], v[36]); v[36] = op.mx(v[32], v[36]); v[32] = t; }
    { uint32_t t = op.mn(v[33], v[37]); v[37] = op.mx(v[33], v[37]); v[33] = t; }
    { uint32_t t = op.mn(v[34], v[38]); v[38] = op.mx(v[34], v[38]); v[34] = t; }
    { uint32_t t = op.mn(v[35], v[39]); v[39] = op.mx(v[35], v[39]); v[35] = t; }
    { uint32_t t = op.mn(v[40], v[44]); v[44] = op.mx(v[40], v[44]); v[40] = t; }
    { uint32_t t = op.mn(v[41], v[45]); v[45] = op.mx(v[41], v[45]); v[41] = t; }
    { uint32_t t = op.mn(v[42], v[46]); v[46] = op.mx(v[42], v[46]); v[42] = t; }
    { uint32_t t = op.mn(v[43], v[47]); v[47] = op.mx(v[43], v[47]); v[43] = t; }
    { uint32_t t = op.mn(v[48], v[52]); v[52] = op.mx(v[48], v[52]); v[48] = t; }
    { uint32_t t = op.mn(v[49], v[53]); v[53] = op.mx(v[49], v[53]); v[49] = t; }
    { uint32_t t = op.mn(v[50], v[54]); v[54] = op.mx(v[50], v[54]); v[50] = t; }
    { uint32_t t = op.mn(v[51], v[55]); v[55] = op.mx(v[51], v[55]); v[51] = t; }
    { uint32_t t = op.mn(v[56], v[60]); v[60] = op.mx(v[56], v[60]); v[56] = t; }
    { uint32_t t = op.mn(v[57], v[61]); v[61] = op.mx(v[57], v[61]); v[57] = t; }
    { uint32_t t = op.mn(v[58], v[62]); v[62] = op.mx(v[58], v[62]); v[58] = t; }
    { uint32_t t = op.mn(v[59], v[63]); v[63] = op.mx(v[59], v[63]); v[59] = t; }
    { uint32_t t = op.mn(v[64], v[68]); v[68] = op.mx(v[64], v[68]); v[64] = t; }
    { uint32_t t = op.mn(v[65], v[69]); v[69] = op.mx(v[65], v[69]); v[65] = t; }
    { uint32_t t = op.mn(v[66], v[70]); v[70] = op.mx(v[66], v[70]); v[66] = t; }
    { uint32_t t = op.mn(v[67], v[71]); v[71] = op.mx(v[67], v[71]); v[67] = t; }
    { uint32_t t = op.mn(v[72], v[76]); v[76] = op.mx(v[72], v[76]); v[72] = t; }
    { uint32_t t = op.mn(v[73], v[77]); v[77] = op.mx(v[73], v[77]); v[73] = t; }
    { uint32_t t = op.mn(v[74], v[78]); v[78] = op.mx(v[74], v[78]); v[74] = t; }
    { uint32_t t = op.mn(v[75], v[79]); v[79] = op.mx(v[75], v[79]); v[75] = t; }
    { uint32_t t = op.mn(v[4], v[64]); v[64] = op.mx(v[4], v[64]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[65]); v[65] = op.mx(v[5], v[65]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[66]); v[66] = op.mx(v[6], v[66]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[67]); v[67] = op.mx(v[7], v[67]); v[7] = t; }
    { uint32_t t = op.mn(v[12], v[72]); v[72] = op.mx(v[12], v[72]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[73]); v[73] = op.mx(v[13], v[73]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[74]); v[74] = op.mx(v[14], v[74]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[75]); v[75] = op.mx(v[15], v[75]); v[15] = t; }
    { uint32_t t = op.mn(v[20], v[80]); v[80] = op.mx(v[20], v[80]); v[20] = t; }
    { uint32_t t = op.mn(v[4], v[32]); v[32] = op.mx(v[4], v[32]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[33]); v[33] = op.mx(v[5], v[33]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[34]); v[34] = op.mx(v[6], v[34]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[35]); v[35] = op.mx(v[7], v[35]); v[7] = t; }
    { uint32_t t = op.mn(v[12], v[40]); v[40] = op.mx(v[12], v[40]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[41]); v[41] = op.mx(v[13], v[41]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[42]); v[42] = op.mx(v[14], v[42]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[43]); v[43] = op.mx(v[15], v[43]); v[15] = t; }
    { uint32_t t = op.mn(v[20], v[48]); v[48] = op.mx(v[20], v[48]); v[20] = t; }
    { uint32_t t = op.mn(v[21], v[49]); v[49] = op.mx(v[21], v[49]); v[21] = t; }
    { uint32_t t = op.mn(v[22], v[50]); v[50] = op.mx(v[22], v[50]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[51]); v[51] = op.mx(v[23], v[51]); v[23] = t; }
    { uint32_t t = op.mn(v[28], v[56]); v[56] = op.mx(v[28], v[56]); v[28] = t; }
    { uint32_t t = op.mn(v[29], v[57]); v[57] = op.mx(v[29], v[57]); v[29] = t; }
    { uint32_t t = op.mn(v[30], v[58]); v[58] = op.mx(v[30], v[58]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[59]); v[59] = op.mx(v[31], v[59]); v[31] = t; }
    { uint32_t t = op.mn(v[36], v[64]); v[64] = op.mx(v[36], v[64]); v[36] = t; }
    { uint32_t t = op.mn(v[37], v[65]); v[65] = op.mx(v[37], v[65]); v[37] = t; }
    { uint32_t t = op.mn(v[38], v[66]); v[66] = op.mx(v[38], v[66]); v[38] = t; }
    { uint32_t t = op.mn(v[39], v[67]); v[67] = op.mx(v[39], v[67]); v[39] = t; }
    { uint32_t t = op.mn(v[44], v[72]); v[72] = op.mx(v[44], v[72]); v[44] = t; }
    { uint32_t t = op.mn(v[45], v[73]); v[73] = op.mx(v[45], v[73]); v[45] = t; }
    { uint32_t t = op.mn(v[46], v[74]); v[74] = op.mx(v[46], v[74]); v[46] = t; }
    { uint32_t t = op.mn(v[47], v[75]); v[75] = op.mx(v[47], v[75]); v[47] = t; }
    { uint32_t t = op.mn(v[52], v[80]); v[80] = op.mx(v[52], v[80]); v[52] = t; }
    { uint32_t t = op.mn(v[4], v[16]); v[16] = op.mx(v[4], v[16]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[17]); v[17] = op.mx(v[5], v[17]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[18]); v[18] = op.mx(v[6], v[18]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[19]); v[19] = op.mx(v[7], v[19]); v[7] = t; }
    { uint32_t t = op.mn(v[12], v[24]); v[24] = op.mx(v[12], v[24]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[25]); v[25] = op.mx(v[13], v[25]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[26]); v[26] = op.mx(v[14], v[26]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[27]); v[27] = op.mx(v[15], v[27]); v[15] = t; }
    { uint32_t t = op.mn(v[20], v[32]); v[32] = op.mx(v[20], v[32]); v[20] = t; }
    { uint32_t t = op.mn(v[21], v[33]); v[33] = op.mx(v[21], v[33]); v[21] = t; }
    { uint32_t t = op.mn(v[22], v[34]); v[34] = op.mx(v[22], v[34]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[35]); v[35] = op.mx(v[23], v[35]); v[23] = t; }
    { uint32_t t = op.mn(v[28], v[40]); v[40] = op.mx(v[28], v[40]); v[28] = t; }
    { uint32_t t = op.mn(v[29], v[41]); v[41] = op.mx(v[29], v[41]); v[29] = t; }
    { uint32_t t = op.mn(v[30], v[42]); v[42] = op.mx(v[30], v[42]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[43]); v[43] = op.mx(v[31], v[43]); v[31] = t; }
    { uint32_t t = op.mn(v[36], v[48]); v[48] = op.mx(v[36], v[48]); v[36] = t; }
    { uint32_t t = op.mn(v[37], v[49]); v[49] = op.mx(v[37], v[49]); v[37] = t; }
    { uint32_t t = op.mn(v[38], v[50]); v[50] = op.mx(v[38], v[50]); v[38] = t; }
    { uint32_t t = op.mn(v[39], v[51]); v[51] = op.mx(v[39], v[51]); v[39] = t; }
    { uint32_t t = op.mn(v[44], v[56]); v[56] = op.mx(v[44], v[56]); v[44] = t; }
    { uint32_t t = op.mn(v[45], v[57]); v[57] = op.mx(v[45], v[57]); v[45] = t; }
    { uint32_t t = op.mn(v[46], v[58]); v[58] = op.mx(v[46], v[58]); v[46] = t; }
    { uint32_t t = op.mn(v[47], v[59]); v[59] = op.mx(v[47], v[59]); v[47] = t; }
    { uint32_t t = op.mn(v[52], v[64]); v[64] = op.mx(v[52], v[64]); v[52] = t; }
    { uint32_t t = op.mn(v[53], v[65]); v[65] = op.mx(v[53], v[65]); v[53] = t; }
    { uint32_t t = op.mn(v[54], v[66]); v[66] = op.mx(v[54], v[66]); v[54] = t; }
    { uint32_t t = op.mn(v[55], v[67]); v[67] = op.mx(v[55], v[67]); v[55] = t; }
    { uint32_t t = op.mn(v[60], v[72]); v[72] = op.mx(v[60], v[72]); v[60] = t; }
    { uint32_t t = op.mn(v[61], v[73]); v[73] = op.mx(v[61], v[73]); v[61] = t; }
    { uint32_t t = op.mn(v[62], v[74]); v[74] = op.mx(v[62], v[74]); v[62] = t; }
    { uint32_t t = op.mn(v[63], v[75]); v[75] = op.mx(v[63], v[75]); v[63] = t; }
    { uint32_t t = op.mn(v[68], v[80]); v[80] = op.mx(v[68], v[80]); v[68] = t; }
    { uint32_t t = op.mn(v[4], v[8]); v[8] = op.mx(v[4], v[8]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[9]); v[9] = op.mx(v[5], v[9]); v[5] = t; }
    { uint32_t t = op.mn(v[6], v[10]); v[10] = op.mx(v[6], v[10]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[11]); v[11] = op.mx(v[7], v[11]); v[7] = t; }
    { uint32_t t = op.mn(v[12], v[16]); v[16] = op.mx(v[12], v[16]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[17]); v[17] = op.mx(v[13], v[17]); v[13] = t; }
    { uint32_t t = op.mn(v[14], v[18]); v[18] = op.mx(v[14], v[18]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[19]); v[19] = op.mx(v[15], v[19]); v[15] = t; }
    { uint32_t t = op.mn(v[20], v[24]); v[24] = op.mx(v[20], v[24]); v[20] = t; }
    { uint32_t t = op.mn(v[21], v[25]); v[25] = op.mx(v[21], v[25]); v[21] = t; }
    { uint32_t t = op.mn(v[22], v[26]); v[26] = op.mx(v[22], v[26]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[27]); v[27] = op.mx(v[23], v[27]); v[23] = t; }
    { uint32_t t = op.mn(v[28], v[32]); v[32] = op.mx(v[28], v[32]); v[28] = t; }
    { uint32_t t = op.mn(v[29], v[33]); v[33] = op.mx(v[29], v[33]); v[29] = t; }
    { uint32_t t = op.mn(v[30], v[34]); v[34] = op.mx(v[30], v[34]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[35]); v[35] = op.mx(v[31], v[35]); v[31] = t; }
    { uint32_t t = op.mn(v[36], v[40]); v[40] = op.mx(v[36], v[40]); v[36] = t; }
    { uint32_t t = op.mn(v[37], v[41]); v[41] = op.mx(v[37], v[41]); v[37] = t; }
    { uint32_t t = op.mn(v[38], v[42]); v[42] = op.mx(v[38], v[42]); v[38] = t; }
    { uint32_t t = op.mn(v[39], v[43]); v[43] = op.mx(v[39], v[43]); v[39] = t; }
    { uint32_t t = op.mn(v[44], v[48]); v[48] = op.mx(v[44], v[48]); v[44] = t; }
    { uint32_t t = op.mn(v[45], v[49]); v[49] = op.mx(v[45], v[49]); v[45] = t; }
    { uint32_t t = op.mn(v[46], v[50]); v[50] = op.mx(v[46], v[50]); v[46] = t; }
    { uint32_t t = op.mn(v[47], v[51]); v[51] = op.mx(v[47], v[51]); v[47] = t; }
    { uint32_t t = op.mn(v[52], v[56]); v[56] = op.mx(v[52], v[56]); v[52] = t; }
    { uint32_t t = op.mn(v[53], v[57]); v[57] = op.mx(v[53], v[57]); v[53] = t; }
    { uint32_t t = op.mn(v[54], v[58]); v[58] = op.mx(v[54], v[58]); v[54] = t; }
    { uint32_t t = op.mn(v[55], v[59]); v[59] = op.mx(v[55], v[59]); v[55] = t; }
    { uint32_t t = op.mn(v[60], v[64]); v[64] = op.mx(v[60], v[64]); v[60] = t; }
    { uint32_t t = op.mn(v[61], v[65]); v[65] = op.mx(v[61], v[65]); v[61] = t; }
    { uint32_t t = op.mn(v[62], v[66]); v[66] = op.mx(v[62], v[66]); v[62] = t; }
    { uint32_t t = op.mn(v[63], v[67]); v[67] = op.mx(v[63], v[67]); v[63] = t; }
    { uint32_t t = op.mn(v[68], v[72]); v[72] = op.mx(v[68], v[72]); v[68] = t; }
    { uint32_t t = op.mn(v[69], v[73]); v[73] = op.mx(v[69], v[73]); v[69] = t; }
    { uint32_t t = op.mn(v[70], v[74]); v[74] = op.mx(v[70], v[74]); v[70] = t; }
    { uint32_t t = op.mn(v[71], v[75]); v[75] = op.mx(v[71], v[75]); v[71] = t; }
    { uint32_t t = op.mn(v[76], v[80]); v[80] = op.mx(v[76], v[80]); v[76] = t; }
    { uint32_t t = op.mn(v[0], v[2]); v[2] = op.mx(v[0], v[2]); v[0] = t; }
    { uint32_t t = op.mn(v[1], v[3]); v[3] = op.mx(v[1], v[3]); v[1] = t; }
    { uint32_t t = op.mn(v[4], v[6]); v[6] = op.mx(v[4], v[6]); v[4] = t; }
    { uint32_t t = op.mn(v[5], v[7]); v[7] = op.mx(v[5], v[7]); v[5] = t; }
    { uint32_t t = op.mn(v[8], v[10]); v[10] = op.mx(v[8], v[10]); v[8] = t; }
    { uint32_t t = op.mn(v[9], v[11]); v[11] = op.mx(v[9], v[11]); v[9] = t; }
    { uint32_t t = op.mn(v[12], v[14]); v[14] = op.mx(v[12], v[14]); v[12] = t; }
    { uint32_t t = op.mn(v[13], v[15]); v[15] = op.mx(v[13], v[15]); v[13] = t; }
    { uint32_t t = op.mn(v[16], v[18]); v[18] = op.mx(v[16], v[18]); v[16] = t; }
    { uint32_t t = op.mn(v[17], v[19]); v[19] = op.mx(v[17], v[19]); v[17] = t; }
    { uint32_t t = op.mn(v[20], v[22]); v[22] = op.mx(v[20], v[22]); v[20] = t; }
    { uint32_t t = op.mn(v[21], v[23]); v[23] = op.mx(v[21], v[23]); v[21] = t; }
    { uint32_t t = op.mn(v[24], v[26]); v[26] = op.mx(v[24], v[26]); v[24] = t; }
    { uint32_t t = op.mn(v[25], v[27]); v[27] = op.mx(v[25], v[27]); v[25] = t; }
    { uint32_t t = op.mn(v[28], v[30]); v[30] = op.mx(v[28], v[30]); v[28] = t; }
    { uint32_t t = op.mn(v[29], v[31]); v[31] = op.mx(v[29], v[31]); v[29] = t; }
    { uint32_t t = op.mn(v[32], v[34]); v[34] = op.mx(v[32], v[34]); v[32] = t; }
    { uint32_t t = op.mn(v[33], v[35]); v[35] = op.mx(v[33], v[35]); v[33] = t; }
    { uint32_t t = op.mn(v[36], v[38]); v[38] = op.mx(v[36], v[38]); v[36] = t; }
    { uint32_t t = op.mn(v[37], v[39]); v[39] = op.mx(v[37], v[39]); v[37] = t; }
    { uint32_t t = op.mn(v[40], v[42]); v[42] = op.mx(v[40], v[42]); v[40] = t; }
    { uint32_t t = op.mn(v[41], v[43]); v[43] = op.mx(v[41], v[43]); v[41] = t; }
    { uint32_t t = op.mn(v[44], v[46]); v[46] = op.mx(v[44], v[46]); v[44] = t; }
    { uint32_t t = op.mn(v[45], v[47]); v[47] = op.mx(v[45], v[47]); v[45] = t; }
    { uint32_t t = op.mn(v[48], v[50]); v[50] = op.mx(v[48], v[50]); v[48] = t; }
    { uint32_t t = op.mn(v[49], v[51]); v[51] = op.mx(v[49], v[51]); v[49] = t; }
    { uint32_t t = op.mn(v[52], v[54]); v[54] = op.mx(v[52], v[54]); v[52] = t; }
    { uint32_t t = op.mn(v[53], v[55]); v[55] = op.mx(v[53], v[55]); v[53] = t; }
    { uint32_t t = op.mn(v[56], v[58]); v[58] = op.mx(v[56], v[58]); v[56] = t; }
    { uint32_t t = op.mn(v[57], v[59]); v[59] = op.mx(v[57], v[59]); v[57] = t; }
    { uint32_t t = op.mn(v[60], v[62]); v[62] = op.mx(v[60], v[62]); v[60] = t; }
    { uint32_t t = op.mn(v[61], v[63]); v[63] = op.mx(v[61], v[63]); v[61] = t; }
    { uint32_t t = op.mn(v[64], v[66]); v[66] = op.mx(v[64], v[66]); v[64] = t; }
    { uint32_t t = op.mn(v[65], v[67]); v[67] = op.mx(v[65], v[67]); v[65] = t; }
    { uint32_t t = op.mn(v[68], v[70]); v[70] = op.mx(v[68], v[70]); v[68] = t; }
    { uint32_t t = op.mn(v[69], v[71]); v[71] = op.mx(v[69], v[71]); v[69] = t; }
    { uint32_t t = op.mn(v[72], v[74]); v[74] = op.mx(v[72], v[74]); v[72] = t; }
    { uint32_t t = op.mn(v[73], v[75]); v[75] = op.mx(v[73], v[75]); v[73] = t; }
    { uint32_t t = op.mn(v[76], v[78]); v[78] = op.mx(v[76], v[78]); v[76] = t; }
    { uint32_t t = op.mn(v[77], v[79]); v[79] = op.mx(v[77], v[79]); v[77] = t; }
    { uint32_t t = op.mn(v[2], v[64]); v[64] = op.mx(v[2], v[64]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[65]); v[65] = op.mx(v[3], v[65]); v[3] = t; }
    { uint32_t t = op.mn(v[6], v[68]); v[68] = op.mx(v[6], v[68]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[69]); v[69] = op.mx(v[7], v[69]); v[7] = t; }
    { uint32_t t = op.mn(v[10], v[72]); v[72] = op.mx(v[10], v[72]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[73]); v[73] = op.mx(v[11], v[73]); v[11] = t; }
    { uint32_t t = op.mn(v[14], v[76]); v[76] = op.mx(v[14], v[76]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[77]); v[77] = op.mx(v[15], v[77]); v[15] = t; }
    { uint32_t t = op.mn(v[18], v[80]); v[80] = op.mx(v[18], v[80]); v[18] = t; }
    { uint32_t t = op.mn(v[2], v[32]); v[32] = op.mx(v[2], v[32]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[33]); v[33] = op.mx(v[3], v[33]); v[3] = t; }
    { uint32_t t = op.mn(v[6], v[36]); v[36] = op.mx(v[6], v[36]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[37]); v[37] = op.mx(v[7], v[37]); v[7] = t; }
    { uint32_t t = op.mn(v[10], v[40]); v[40] = op.mx(v[10], v[40]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[41]); v[41] = op.mx(v[11], v[41]); v[11] = t; }
    { uint32_t t = op.mn(v[14], v[44]); v[44] = op.mx(v[14], v[44]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[45]); v[45] = op.mx(v[15], v[45]); v[15] = t; }
    { uint32_t t = op.mn(v[18], v[48]); v[48] = op.mx(v[18], v[48]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[49]); v[49] = op.mx(v[19], v[49]); v[19] = t; }
    { uint32_t t = op.mn(v[22], v[52]); v[52] = op.mx(v[22], v[52]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[53]); v[53] = op.mx(v[23], v[53]); v[23] = t; }
    { uint32_t t = op.mn(v[26], v[56]); v[56] = op.mx(v[26], v[56]); v[26] = t; }
    { uint32_t t = op.mn(v[27], v[57]); v[57] = op.mx(v[27], v[57]); v[27] = t; }
    { uint32_t t = op.mn(v[30], v[60]); v[60] = op.mx(v[30], v[60]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[61]); v[61] = op.mx(v[31], v[61]); v[31] = t; }
    { uint32_t t = op.mn(v[34], v[64]); v[64] = op.mx(v[34], v[64]); v[34] = t; }
    { uint32_t t = op.mn(v[35], v[65]); v[65] = op.mx(v[35], v[65]); v[35] = t; }
    { uint32_t t = op.mn(v[38], v[68]); v[68] = op.mx(v[38], v[68]); v[38] = t; }
    { uint32_t t = op.mn(v[39], v[69]); v[69] = op.mx(v[39], v[69]); v[39] = t; }
    { uint32_t t = op.mn(v[42], v[72]); v[72] = op.mx(v[42], v[72]); v[42] = t; }
    { uint32_t t = op.mn(v[43], v[73]); v[73] = op.mx(v[43], v[73]); v[43] = t; }
    { uint32_t t = op.mn(v[46], v[76]); v[76] = op.mx(v[46], v[76]); v[46] = t; }
    { uint32_t t = op.mn(v[47], v[77]); v[77] = op.mx(v[47], v[77]); v[47] = t; }
    { uint32_t t = op.mn(v[50], v[80]); v[80] = op.mx(v[50], v[80]); v[50] = t; }
    { uint32_t t = op.mn(v[2], v[16]); v[16] = op.mx(v[2], v[16]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[17]); v[17] = op.mx(v[3], v[17]); v[3] = t; }
    { uint32_t t = op.mn(v[6], v[20]); v[20] = op.mx(v[6], v[20]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[21]); v[21] = op.mx(v[7], v[21]); v[7] = t; }
    { uint32_t t = op.mn(v[10], v[24]); v[24] = op.mx(v[10], v[24]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[25]); v[25] = op.mx(v[11], v[25]); v[11] = t; }
    { uint32_t t = op.mn(v[14], v[28]); v[28] = op.mx(v[14], v[28]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[29]); v[29] = op.mx(v[15], v[29]); v[15] = t; }
    { uint32_t t = op.mn(v[18], v[32]); v[32] = op.mx(v[18], v[32]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[33]); v[33] = op.mx(v[19], v[33]); v[19] = t; }
    { uint32_t t = op.mn(v[22], v[36]); v[36] = op.mx(v[22], v[36]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[37]); v[37] = op.mx(v[23], v[37]); v[23] = t; }
    { uint32_t t = op.mn(v[26], v[40]); v[40] = op.mx(v[26], v[40]); v[26] = t; }
    { uint32_t t = op.mn(v[27], v[41]); v[41] = op.mx(v[27], v[41]); v[27] = t; }
    { uint32_t t = op.mn(v[30], v[44]); v[44] = op.mx(v[30], v[44]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[45]); v[45] = op.mx(v[31], v[45]); v[31] = t; }
    { uint32_t t = op.mn(v[34], v[48]); v[48] = op.mx(v[34], v[48]); v[34] = t; }
    { uint32_t t = op.mn(v[35], v[49]); v[49] = op.mx(v[35], v[49]); v[35] = t; }
    { uint32_t t = op.mn(v[38], v[52]); v[52] = op.mx(v[38], v[52]); v[38] = t; }
    { uint32_t t = op.mn(v[39], v[53]); v[53] = op.mx(v[39], v[53]); v[39] = t; }
    { uint32_t t = op.mn(v[42], v[56]); v[56] = op.mx(v[42], v[56]); v[42] = t; }
    { uint32_t t = op.mn(v[43], v[57]); v[57] = op.mx(v[43], v[57]); v[43] = t; }
    { uint32_t t = op.mn(v[46], v[60]); v[60] = op.mx(v[46], v[60]); v[46] = t; }
    { uint32_t t = op.mn(v[47], v[61]); v[61] = op.mx(v[47], v[61]); v[47] = t; }
    { uint32_t t = op.mn(v[50], v[64]); v[64] = op.mx(v[50], v[64]); v[50] = t; }
    { uint32_t t = op.mn(v[51], v[65]); v[65] = op.mx(v[51], v[65]); v[51] = t; }
    { uint32_t t = op.mn(v[54], v[68]); v[68] = op.mx(v[54], v[68]); v[54] = t; }
    { uint32_t t = op.mn(v[55], v[69]); v[69] = op.mx(v[55], v[69]); v[55] = t; }
    { uint32_t t = op.mn(v[58], v[72]); v[72] = op.mx(v[58], v[72]); v[58] = t; }
    { uint32_t t = op.mn(v[59], v[73]); v[73] = op.mx(v[59], v[73]); v[59] = t; }
    { uint32_t t = op.mn(v[62], v[76]); v[76] = op.mx(v[62], v[76]); v[62] = t; }
    { uint32_t t = op.mn(v[63], v[77]); v[77] = op.mx(v[63], v[77]); v[63] = t; }
    { uint32_t t = op.mn(v[66], v[80]); v[80] = op.mx(v[66], v[80]); v[66] = t; }
    { uint32_t t = op.mn(v[2], v[8]); v[8] = op.mx(v[2], v[8]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[9]); v[9] = op.mx(v[3], v[9]); v[3] = t; }
    { uint32_t t = op.mn(v[6], v[12]); v[12] = op.mx(v[6], v[12]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[13]); v[13] = op.mx(v[7], v[13]); v[7] = t; }
    { uint32_t t = op.mn(v[10], v[16]); v[16] = op.mx(v[10], v[16]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[17]); v[17] = op.mx(v[11], v[17]); v[11] = t; }
    { uint32_t t = op.mn(v[14], v[20]); v[20] = op.mx(v[14], v[20]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[21]); v[21] = op.mx(v[15], v[21]); v[15] = t; }
    { uint32_t t = op.mn(v[18], v[24]); v[24] = op.mx(v[18], v[24]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[25]); v[25] = op.mx(v[19], v[25]); v[19] = t; }
    { uint32_t t = op.mn(v[22], v[28]); v[28] = op.mx(v[22], v[28]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[29]); v[29] = op.mx(v[23], v[29]); v[23] = t; }
    { uint32_t t = op.mn(v[26], v[32]); v[32] = op.mx(v[26], v[32]); v[26] = t; }
    { uint32_t t = op.mn(v[27], v[33]); v[33] = op.mx(v[27], v[33]); v[27] = t; }
    { uint32_t t = op.mn(v[30], v[36]); v[36] = op.mx(v[30], v[36]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[37]); v[37] = op.mx(v[31], v[37]); v[31] = t; }
    { uint32_t t = op.mn(v[34], v[40]); v[40] = op.mx(v[34], v[40]); v[34] = t; }
    { uint32_t t = op.mn(v[35], v[41]); v[41] = op.mx(v[35], v[41]); v[35] = t; }
    { uint32_t t = op.mn(v[38], v[44]); v[44] = op.mx(v[38], v[44]); v[38] = t; }
    { uint32_t t = op.mn(v[39], v[45]); v[45] = op.mx(v[39], v[45]); v[39] = t; }
    { uint32_t t = op.mn(v[42], v[48]); v[48] = op.mx(v[42], v[48]); v[42] = t; }
    { uint32_t t = op.mn(v[43], v[49]); v[49] = op.mx(v[43], v[49]); v[43] = t; }
    { uint32_t t = op.mn(v[46], v[52]); v[52] = op.mx(v[46], v[52]); v[46] = t; }
    { uint32_t t = op.mn(v[47], v[53]); v[53] = op.mx(v[47], v[53]); v[47] = t; }
    { uint32_t t = op.mn(v[50], v[56]); v[56] = op.mx(v[50], v[56]); v[50] = t; }
    { uint32_t t = op.mn(v[51], v[57]); v[57] = op.mx(v[51], v[57]); v[51] = t; }
    { uint32_t t = op.mn(v[54], v[60]); v[60] = op.mx(v[54], v[60]); v[54] = t; }
    { uint32_t t = op.mn(v[55], v[61]); v[61] = op.mx(v[55], v[61]); v[55] = t; }
    { uint32_t t = op.mn(v[58], v[64]); v[64] = op.mx(v[58], v[64]); v[58] = t; }
    { uint32_t t = op.mn(v[59], v[65]); v[65] = op.mx(v[59], v[65]); v[59] = t; }
    { uint32_t t = op.mn(v[62], v[68]); v[68] = op.mx(v[62], v[68]); v[62] = t; }
    { uint32_t t = op.mn(v[63], v[69]); v[69] = op.mx(v[63], v[69]); v[63] = t; }
    { uint32_t t = op.mn(v[66], v[72]); v[72] = op.mx(v[66], v[72]); v[66] = t; }
    { uint32_t t = op.mn(v[67], v[73]); v[73] = op.mx(v[67], v[73]); v[67] = t; }
    { uint32_t t = op.mn(v[70], v[76]); v[76] = op.mx(v[70], v[76]); v[70] = t; }
    { uint32_t t = op.mn(v[71], v[77]); v[77] = op.mx(v[71], v[77]); v[71] = t; }
    { uint32_t t = op.mn(v[74], v[80]); v[80] = op.mx(v[74], v[80]); v[74] = t; }
    { uint32_t t = op.mn(v[2], v[4]); v[4] = op.mx(v[2], v[4]); v[2] = t; }
    { uint32_t t = op.mn(v[3], v[5]); v[5] = op.mx(v[3], v[5]); v[3] = t; }
    { uint32_t t = op.mn(v[6], v[8]); v[8] = op.mx(v[6], v[8]); v[6] = t; }
    { uint32_t t = op.mn(v[7], v[9]); v[9] = op.mx(v[7], v[9]); v[7] = t; }
    { uint32_t t = op.mn(v[10], v[12]); v[12] = op.mx(v[10], v[12]); v[10] = t; }
    { uint32_t t = op.mn(v[11], v[13]); v[13] = op.mx(v[11], v[13]); v[11] = t; }
    { uint32_t t = op.mn(v[14], v[16]); v[16] = op.mx(v[14], v[16]); v[14] = t; }
    { uint32_t t = op.mn(v[15], v[17]); v[17] = op.mx(v[15], v[17]); v[15] = t; }
    { uint32_t t = op.mn(v[18], v[20]); v[20] = op.mx(v[18], v[20]); v[18] = t; }
    { uint32_t t = op.mn(v[19], v[21]); v[21] = op.mx(v[19], v[21]); v[19] = t; }
    { uint32_t t = op.mn(v[22], v[24]); v[24] = op.mx(v[22], v[24]); v[22] = t; }
    { uint32_t t = op.mn(v[23], v[25]); v[25] = op.mx(v[23], v[25]); v[23] = t; }
    { uint32_t t = op.mn(v[26], v[28]); v[28] = op.mx(v[26], v[28]); v[26] = t; }
    { uint32_t t = op.mn(v[27], v[29]); v[29] = op.mx(v[27], v[29]); v[27] = t; }
    { uint32_t t = op.mn(v[30], v[32]); v[32] = op.mx(v[30], v[32]); v[30] = t; }
    { uint32_t t = op.mn(v[31], v[33]); v[33] = op.mx(v[31], v[33]); v[31] = t; }
    { uint32_t t = op.mn(v[34], v[36]); v[36] = op.mx(v[34], v[36]); v[34] = t; }
    { uint32_t t = op.mn(v[35], v[37]); v[37] = op.mx(v[35], v[37]); v[35] = t; }
    { uint32_t t = op.mn(v[38], v[40]); v[40] = op.mx(v[38], v[40]); v[38] = t; }
    { uint32_t t = op.mn(v[39], v[41]); v[41] = op.mx(v[39], v[41]); v[39] = t; }
    { uint32_t t = op.mn(v[42], v[44]); v[44] = op.mx(v[42], v[44]); v[42] = t; }
    { uint32_t t = op.mn(v[43], v[45]); v[45] = op.mx(v[43], v[45]); v[43] = t; }
    { uint32_t t = op.mn(v[46], v[48]); v[48] = op.mx(v[46], v[48]); v[46] = t; }
    { uint32_t t = op.mn(v[47], v[49]); v[49] = op.mx(v[47], v[49]); v[47] = t; }
    { uint32_t t = op.mn(v[50], v[52]); v[52] = op.mx(v[50], v[52]); v[50] = t; }
    { uint32_t t = op.mn(v[51], v[53]); v[53] = op.mx(v[51], v[53]); v[51] = t; }
    { uint32_t t = op.mn(v[54], v[56]); v[56] = op.mx(v[54], v[56]); v[54] = t; }
    { uint32_t t = op.mn(v[55], v[57]); v[57] = op.mx(v[55], v[57]); v[55] = t; }
    { uint32_t t = op.mn(v[58], v[60]); v[60] = op.mx(v[58], v[60]); v[58] = t; }
    { uint32_t t = op.mn(v[59], v[61]); v[61] = op.mx(v[59], v[61]); v[59] = t; }
    { uint32_t t = op.mn(v[62], v[64]); v[64] = op.mx(v[62], v[64]); v[62] = t; }
    { uint32_t t = op.mn(v[63], v[65]); v[65] = op.mx(v[63], v[65]); v[63] = t; }
    { uint32_t t = op.mn(v[66], v[68]); v[68] = op.mx(v[66], v[68]); v[66] = t; }
    { uint32_t t = op.mn(v[67], v[69]); v[69] = op.mx(v[67], v[69]); v[67] = t; }
    { uint32_t t = op.mn(v[70], v[72]); v[72] = op.mx(v[70], v[72]); v[70] = t; }
    { uint32_t t = op.mn(v[71], v[73]); v[73] = op.mx(v[71], v[73]); v[71] = t; }
    { uint32_t t = op.mn(v[74], v[76]); v[76] = op.mx(v[74], v[76]); v[74] = t; }
    { uint32_t t = op.mn(v[75], v[77]); v[77] = op.mx(v[75], v[77]); v[75] = t; }
    { uint32_t t = op.mn(v[78], v[80]); v[80] = op.mx(v[78], v[80]); v[78] = t; }
    v[1] = op.mx(v[0], v[1]);
    v[3] = op.mx(v[2], v[3]);
    v[5] = op.mx(v[4], v[5]);
    v[7] = op.mx(v[6], v[7]);
    v[9] = op.mx(v[8], v[9]);
    v[11] = op.mx(v[10], v[11]);
    v[13] = op.mx(v[12], v[13]);
    v[15] = op.mx(v[14], v[15]);
    v[17] = op.mx(v[16], v[17]);
    v[19] = op.mx(v[18], v[19]);
    v[21] = op.mx(v[20], v[21]);
    v[23] = op.mx(v[22], v[23]);
    v[25] = op.mx(v[24], v[25]);
    v[27] = op.mx(v[26], v[27]);
    v[29] = op.mx(v[28], v[29]);
    v[31] = op.mx(v[30], v[31]);
    v[33] = op.mx(v[32], v[33]);
    v[35] = op.mx(v[34], v[35]);
    v[37] = op.mx(v[36], v[37]);
    v[39] = op.mx(v[38], v[39]);
    v[40] = op.mn(v[40], v[41]);
    v[42] = op.mn(v[42], v[43]);
    v[44] = op.mn(v[44], v[45]);
    v[46] = op.mn(v[46], v[47]);
    v[48] = op.mn(v[48], v[49]);
    v[50] = op.mn(v[50], v[51]);
    v[52] = op.mn(v[52], v[53]);
    v[54] = op.mn(v[54], v[55]);
    v[56] = op.mn(v[56], v[57]);
    v[58] = op.mn(v[58], v[59]);
    v[60] = op.mn(v[60], v[61]);
    v[62] = op.mn(v[62], v[63]);
    v[64] = op.mn(v[64], v[65]);
    v[66] = op.mn(v[66], v[67]);
    v[68] = op.mn(v[68], v[69]);
    v[70] = op.mn(v[70], v[71]);
    v[72] = op.mn(v[72], v[73]);
    v[74] = op.mn(v[74], v[75]);
    v[76] = op.mn(v[76], v[77]);
    v[78] = op.mn(v[78], v[79]);
    v[64] = op.mx(v[1], v[64]);
    v[66] = op.mx(v[3], v[66]);
    v[68] = op.mx(v[5], v[68]);
    v[70] = op.mx(v[7], v[70]);
    v[9] = op.mn(v[9], v[72]);
    v[11] = op.mn(v[11], v[74]);
    v[13] = op.mn(v[13], v[76]);
    v[15] = op.mn(v[15], v[78]);
    v[17] = op.mn(v[17], v[80]);
    v[40] = op.mx(v[9], v[40]);
    v[42] = op.mx(v[11], v[42]);
    v[44] = op.mx(v[13], v[44]);
    v[46] = op.mx(v[15], v[46]);
    v[48] = op.mx(v[17], v[48]);
    v[50] = op.mx(v[19], v[50]);
    v[52] = op.mx(v[21], v[52]);
    v[54] = op.mx(v[23], v[54]);
    v[25] = op.mn(v[25], v[56]);
    v[27] = op.mn(v[27], v[58]);
    v[29] = op.mn(v[29], v[60]);
    v[31] = op.mn(v[31], v[62]);
    v[33] = op.mn(v[33], v[64]);
    v[35] = op.mn(v[35], v[66]);
    v[37] = op.mn(v[37], v[68]);
    v[39] = op.mn(v[39], v[70]);
    v[40] = op.mx(v[25], v[40]);
    v[42] = op.mx(v[27], v[42]);
    v[44] = op.mx(v[29], v[44]);
    v[46] = op.mx(v[31], v[46]);
    v[33] = op.mn(v[33], v[48]);
    v[35] = op.mn(v[35], v[50]);
    v[37] = op.mn(v[37], v[52]);
    v[39] = op.mn(v[39], v[54]);
    v[40] = op.mx(v[33], v[40]);
    v[42] = op.mx(v[35], v[42]);
    v[37] = op.mn(v[37], v[44]);
    v[39] = op.mn(v[39], v[46]);
    v[40] = op.mx(v[37], v[40]);
    v[39] = op.mn(v[39], v[42]);
    v[40] = op.mx(v[39], v[40]);
    return v[40];
  }
};

}  // namespace fnr
