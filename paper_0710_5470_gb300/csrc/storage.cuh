// Storage formats of the populations in HBM.
//
//   StF64   f_i in float64, arithmetic in float64;
//   StF32   f_i in float32, arithmetic in float32;
//   StF16   f_0 in float32, f_i - fref_i (i >= 1) in fp16, arithmetic float32;
//   StBF16  f_0 in float32, f_i - fref_i (i >= 1) in bf16, arithmetic float32.
// fref_i = w_i p0(rho_ref) is the rest equilibrium of Eq. 5 (u = 0, zero
// gradients); bulk liquid and gas at coexistence share p0, so the stored
// deviations are small away from interfaces.  f_0 carries the O(1) density
// contrast between the phases and stays float32.
//
// Populations are separate arrays (structure of arrays), one pointer each.
// The x2 forms move two adjacent sites (even element index q, arrays
// 256-byte aligned) with one 2-vector access.
// The step kernels work on deviations d_i = f_i - fref_i (i >= 1; fref = 0
// for StF64 / StF32): devi / sti read and write the stored deviation, f_0 is
// stored as is.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace lbk {

struct StF64 {
    using real = double;
    using raw0 = double;   // stored type of f_0
    using rawi = double;   // stored type of f_i, i >= 1
    using raw0x2 = double2;   // two adjacent sites (element index even)
    using rawix2 = double2;
    static constexpr int id = 0;
    __device__ __forceinline__ static raw0x2 ld0x2(const char* p, size_t q) { return reinterpret_cast<const double2*>(p)[q >> 1]; }
    __device__ __forceinline__ static rawix2 ldix2(const char* p, size_t q) { return reinterpret_cast<const double2*>(p)[q >> 1]; }
    __device__ __forceinline__ static void dec0x2(raw0x2 v, real& a, real& b) { a = v.x; b = v.y; }
    __device__ __forceinline__ static void devix2(rawix2 v, real& a, real& b) { a = v.x; b = v.y; }
    __device__ __forceinline__ static raw0 ld0(const char* p, size_t idx) { return reinterpret_cast<const double*>(p)[idx]; }
    __device__ __forceinline__ static rawi ldi(const char* p, size_t idx) { return reinterpret_cast<const double*>(p)[idx]; }
    __device__ __forceinline__ static real dec0(raw0 v) { return v; }
    __device__ __forceinline__ static real deci(rawi v, float) { return v; }
    __device__ __forceinline__ static real devi(rawi v) { return v; }
    __device__ __forceinline__ static void st0(char* p, size_t idx, real v) { reinterpret_cast<double*>(p)[idx] = v; }
    __device__ __forceinline__ static void sti(char* p, size_t idx, real d) { reinterpret_cast<double*>(p)[idx] = d; }
    __host__ __device__ static constexpr int bytes(int) { return 8; }
    __host__ __device__ static constexpr long long pop_offset(int i, long long pitch) { return i * pitch * 8; }
    __device__ __forceinline__ static real load(int, const char* p, size_t idx, float) {
        return reinterpret_cast<const double*>(p)[idx];
    }
    __device__ __forceinline__ static void store(int, char* p, size_t idx, real v, float) {
        reinterpret_cast<double*>(p)[idx] = v;
    }
};

struct StF32 {
    using real = float;
    using raw0 = float;
    using rawi = float;
    using raw0x2 = float2;
    using rawix2 = float2;
    static constexpr int id = 1;
    __device__ __forceinline__ static raw0x2 ld0x2(const char* p, size_t q) { return reinterpret_cast<const float2*>(p)[q >> 1]; }
    __device__ __forceinline__ static rawix2 ldix2(const char* p, size_t q) { return reinterpret_cast<const float2*>(p)[q >> 1]; }
    __device__ __forceinline__ static void dec0x2(raw0x2 v, real& a, real& b) { a = v.x; b = v.y; }
    __device__ __forceinline__ static void devix2(rawix2 v, real& a, real& b) { a = v.x; b = v.y; }
    __device__ __forceinline__ static raw0 ld0(const char* p, size_t idx) { return reinterpret_cast<const float*>(p)[idx]; }
    __device__ __forceinline__ static rawi ldi(const char* p, size_t idx) { return reinterpret_cast<const float*>(p)[idx]; }
    __device__ __forceinline__ static real dec0(raw0 v) { return v; }
    __device__ __forceinline__ static real deci(rawi v, float) { return v; }
    __device__ __forceinline__ static real devi(rawi v) { return v; }
    __device__ __forceinline__ static void st0(char* p, size_t idx, real v) { reinterpret_cast<float*>(p)[idx] = v; }
    __device__ __forceinline__ static void sti(char* p, size_t idx, real d) { reinterpret_cast<float*>(p)[idx] = d; }
    __host__ __device__ static constexpr int bytes(int) { return 4; }
    __host__ __device__ static constexpr long long pop_offset(int i, long long pitch) { return i * pitch * 4; }
    __device__ __forceinline__ static real load(int, const char* p, size_t idx, float) {
        return reinterpret_cast<const float*>(p)[idx];
    }
    __device__ __forceinline__ static void store(int, char* p, size_t idx, real v, float) {
        reinterpret_cast<float*>(p)[idx] = v;
    }
};

struct StF16 {
    using real = float;
    using raw0 = float;
    using rawi = __half;
    using raw0x2 = float2;
    using rawix2 = __half2;
    static constexpr int id = 2;
    __device__ __forceinline__ static raw0x2 ld0x2(const char* p, size_t q) { return reinterpret_cast<const float2*>(p)[q >> 1]; }
    __device__ __forceinline__ static rawix2 ldix2(const char* p, size_t q) { return reinterpret_cast<const __half2*>(p)[q >> 1]; }
    __device__ __forceinline__ static void dec0x2(raw0x2 v, real& a, real& b) { a = v.x; b = v.y; }
    __device__ __forceinline__ static void devix2(rawix2 v, real& a, real& b) {
        a = __low2float(v);
        b = __high2float(v);
    }
    __device__ __forceinline__ static raw0 ld0(const char* p, size_t idx) { return reinterpret_cast<const float*>(p)[idx]; }
    __device__ __forceinline__ static rawi ldi(const char* p, size_t idx) { return reinterpret_cast<const __half*>(p)[idx]; }
    __device__ __forceinline__ static real dec0(raw0 v) { return v; }
    __device__ __forceinline__ static real deci(rawi v, float ref) { return __half2float(v) + ref; }
    __device__ __forceinline__ static real devi(rawi v) { return __half2float(v); }
    __device__ __forceinline__ static void st0(char* p, size_t idx, real v) { reinterpret_cast<float*>(p)[idx] = v; }
    __device__ __forceinline__ static void sti(char* p, size_t idx, real d) {
        reinterpret_cast<__half*>(p)[idx] = __float2half_rn(d);
    }
    __host__ __device__ static constexpr int bytes(int i) { return i == 0 ? 4 : 2; }
    __host__ __device__ static constexpr long long pop_offset(int i, long long pitch) {
        return i == 0 ? 0 : pitch * 4 + (i - 1) * pitch * 2;
    }
    __device__ __forceinline__ static real load(int i, const char* p, size_t idx, float ref) {
        if (i == 0) return reinterpret_cast<const float*>(p)[idx];
        return __half2float(reinterpret_cast<const __half*>(p)[idx]) + ref;
    }
    __device__ __forceinline__ static void store(int i, char* p, size_t idx, real v, float ref) {
        if (i == 0) {
            reinterpret_cast<float*>(p)[idx] = v;
            return;
        }
        reinterpret_cast<__half*>(p)[idx] = __float2half_rn(v - ref);
    }
};

struct StBF16 {
    using real = float;
    using raw0 = float;
    using rawi = __nv_bfloat16;
    using raw0x2 = float2;
    using rawix2 = __nv_bfloat162;
    static constexpr int id = 3;
    __device__ __forceinline__ static raw0x2 ld0x2(const char* p, size_t q) { return reinterpret_cast<const float2*>(p)[q >> 1]; }
    __device__ __forceinline__ static rawix2 ldix2(const char* p, size_t q) {
        return reinterpret_cast<const __nv_bfloat162*>(p)[q >> 1];
    }
    __device__ __forceinline__ static void dec0x2(raw0x2 v, real& a, real& b) { a = v.x; b = v.y; }
    __device__ __forceinline__ static void devix2(rawix2 v, real& a, real& b) {
        a = __low2float(v);
        b = __high2float(v);
    }
    __device__ __forceinline__ static raw0 ld0(const char* p, size_t idx) { return reinterpret_cast<const float*>(p)[idx]; }
    __device__ __forceinline__ static rawi ldi(const char* p, size_t idx) {
        return reinterpret_cast<const __nv_bfloat16*>(p)[idx];
    }
    __device__ __forceinline__ static real dec0(raw0 v) { return v; }
    __device__ __forceinline__ static real deci(rawi v, float ref) { return __bfloat162float(v) + ref; }
    __device__ __forceinline__ static real devi(rawi v) { return __bfloat162float(v); }
    __device__ __forceinline__ static void st0(char* p, size_t idx, real v) { reinterpret_cast<float*>(p)[idx] = v; }
    __device__ __forceinline__ static void sti(char* p, size_t idx, real d) {
        reinterpret_cast<__nv_bfloat16*>(p)[idx] = __float2bfloat16_rn(d);
    }
    __host__ __device__ static constexpr int bytes(int i) { return i == 0 ? 4 : 2; }
    __host__ __device__ static constexpr long long pop_offset(int i, long long pitch) {
        return i == 0 ? 0 : pitch * 4 + (i - 1) * pitch * 2;
    }
    __device__ __forceinline__ static real load(int i, const char* p, size_t idx, float ref) {
        if (i == 0) return reinterpret_cast<const float*>(p)[idx];
        return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[idx]) + ref;
    }
    __device__ __forceinline__ static void store(int i, char* p, size_t idx, real v, float ref) {
        if (i == 0) {
            reinterpret_cast<float*>(p)[idx] = v;
            return;
        }
        reinterpret_cast<__nv_bfloat16*>(p)[idx] = __float2bfloat16_rn(v - ref);
    }
};

}  // namespace lbk
