/* Generated by gen_tables.py -- exact constants for the Falcon kernels. */
#pragma once
#include <stdint.h>

#ifndef FALCON_TABLE_QUAL
#define FALCON_TABLE_QUAL static const
#endif

#define FALCON_P10_F64_LO (-30)
#define FALCON_P10_F64_HI (22)
#define FALCON_P10_F32_LO (-15)
#define FALCON_P10_F32_HI (10)
#define FALCON_P10_F16_LO (-8)
#define FALCON_P10_F16_HI (4)

FALCON_TABLE_QUAL uint64_t FALCON_POW5[23] = {
    0x0000000000000001ull, /* 5^0 */
    0x0000000000000005ull, /* 5^1 */
    0x0000000000000019ull, /* 5^2 */
    0x000000000000007dull, /* 5^3 */
    0x0000000000000271ull, /* 5^4 */
    0x0000000000000c35ull, /* 5^5 */
    0x0000000000003d09ull, /* 5^6 */
    0x000000000001312dull, /* 5^7 */
    0x000000000005f5e1ull, /* 5^8 */
    0x00000000001dcd65ull, /* 5^9 */
    0x00000000009502f9ull, /* 5^10 */
    0x0000000002e90eddull, /* 5^11 */
    0x000000000e8d4a51ull, /* 5^12 */
    0x0000000048c27395ull, /* 5^13 */
    0x000000016bcc41e9ull, /* 5^14 */
    0x000000071afd498dull, /* 5^15 */
    0x0000002386f26fc1ull, /* 5^16 */
    0x000000b1a2bc2ec5ull, /* 5^17 */
    0x000003782dace9d9ull, /* 5^18 */
    0x00001158e460913dull, /* 5^19 */
    0x000056bc75e2d631ull, /* 5^20 */
    0x0001b1ae4d6e2ef5ull, /* 5^21 */
    0x000878678326eac9ull, /* 5^22 */
};

FALCON_TABLE_QUAL uint64_t FALCON_RECIP5[23] = {
    0x0000000000000000ull, /* 5^0 */
    0xccccccccccccccccull, /* 5^1 */
    0xa3d70a3d70a3d70aull, /* 5^2 */
    0x83126e978d4fdf3bull, /* 5^3 */
    0xd1b71758e219652bull, /* 5^4 */
    0xa7c5ac471b478423ull, /* 5^5 */
    0x8637bd05af6c69b5ull, /* 5^6 */
    0xd6bf94d5e57a42bcull, /* 5^7 */
    0xabcc77118461cefcull, /* 5^8 */
    0x89705f4136b4a597ull, /* 5^9 */
    0xdbe6fecebdedd5beull, /* 5^10 */
    0xafebff0bcb24aafeull, /* 5^11 */
    0x8cbccc096f5088cbull, /* 5^12 */
    0xe12e13424bb40e13ull, /* 5^13 */
    0xb424dc35095cd80full, /* 5^14 */
    0x901d7cf73ab0acd9ull, /* 5^15 */
    0xe69594bec44de15bull, /* 5^16 */
    0xb877aa3236a4b449ull, /* 5^17 */
    0x9392ee8e921d5d07ull, /* 5^18 */
    0xec1e4a7db69561a5ull, /* 5^19 */
    0xbce5086492111aeaull, /* 5^20 */
    0x971da05074da7beeull, /* 5^21 */
    0xf1c90080baf72cb1ull, /* 5^22 */
};

FALCON_TABLE_QUAL uint64_t FALCON_POW5_NORM[23] = {
    0x8000000000000000ull, /* 5^0 */
    0xa000000000000000ull, /* 5^1 */
    0xc800000000000000ull, /* 5^2 */
    0xfa00000000000000ull, /* 5^3 */
    0x9c40000000000000ull, /* 5^4 */
    0xc350000000000000ull, /* 5^5 */
    0xf424000000000000ull, /* 5^6 */
    0x9896800000000000ull, /* 5^7 */
    0xbebc200000000000ull, /* 5^8 */
    0xee6b280000000000ull, /* 5^9 */
    0x9502f90000000000ull, /* 5^10 */
    0xba43b74000000000ull, /* 5^11 */
    0xe8d4a51000000000ull, /* 5^12 */
    0x9184e72a00000000ull, /* 5^13 */
    0xb5e620f480000000ull, /* 5^14 */
    0xe35fa931a0000000ull, /* 5^15 */
    0x8e1bc9bf04000000ull, /* 5^16 */
    0xb1a2bc2ec5000000ull, /* 5^17 */
    0xde0b6b3a76400000ull, /* 5^18 */
    0x8ac7230489e80000ull, /* 5^19 */
    0xad78ebc5ac620000ull, /* 5^20 */
    0xd8d726b7177a8000ull, /* 5^21 */
    0x878678326eac9000ull, /* 5^22 */
};

FALCON_TABLE_QUAL uint8_t FALCON_LOG2_POW5[23] = {
    0, 2, 4, 6, 9, 11, 13, 16, 18, 20, 23, 25, 27, 30, 32, 34, 37, 39, 41, 44, 46, 48, 51
};

FALCON_TABLE_QUAL uint64_t FALCON_P10_F64[53] = {
    0x39b4484bfeebc2a0ull, /* fl64(1e-30) */
    0x39e95a5efea6b347ull, /* fl64(1e-29) */
    0x3a1fb0f6be506019ull, /* fl64(1e-28) */
    0x3a53ce9a36f23c10ull, /* fl64(1e-27) */
    0x3a88c240c4aecb14ull, /* fl64(1e-26) */
    0x3abef2d0f5da7dd9ull, /* fl64(1e-25) */
    0x3af357c299a88ea7ull, /* fl64(1e-24) */
    0x3b282db34012b251ull, /* fl64(1e-23) */
    0x3b5e392010175ee6ull, /* fl64(1e-22) */
    0x3b92e3b40a0e9b4full, /* fl64(1e-21) */
    0x3bc79ca10c924223ull, /* fl64(1e-20) */
    0x3bfd83c94fb6d2acull, /* fl64(1e-19) */
    0x3c32725dd1d243acull, /* fl64(1e-18) */
    0x3c670ef54646d497ull, /* fl64(1e-17) */
    0x3c9cd2b297d889bcull, /* fl64(1e-16) */
    0x3cd203af9ee75616ull, /* fl64(1e-15) */
    0x3d06849b86a12b9bull, /* fl64(1e-14) */
    0x3d3c25c268497682ull, /* fl64(1e-13) */
    0x3d719799812dea11ull, /* fl64(1e-12) */
    0x3da5fd7fe1796495ull, /* fl64(1e-11) */
    0x3ddb7cdfd9d7bdbbull, /* fl64(1e-10) */
    0x3e112e0be826d695ull, /* fl64(1e-9) */
    0x3e45798ee2308c3aull, /* fl64(1e-8) */
    0x3e7ad7f29abcaf48ull, /* fl64(1e-7) */
    0x3eb0c6f7a0b5ed8dull, /* fl64(1e-6) */
    0x3ee4f8b588e368f1ull, /* fl64(1e-5) */
    0x3f1a36e2eb1c432dull, /* fl64(1e-4) */
    0x3f50624dd2f1a9fcull, /* fl64(1e-3) */
    0x3f847ae147ae147bull, /* fl64(1e-2) */
    0x3fb999999999999aull, /* fl64(1e-1) */
    0x3ff0000000000000ull, /* fl64(1e0) */
    0x4024000000000000ull, /* fl64(1e1) */
    0x4059000000000000ull, /* fl64(1e2) */
    0x408f400000000000ull, /* fl64(1e3) */
    0x40c3880000000000ull, /* fl64(1e4) */
    0x40f86a0000000000ull, /* fl64(1e5) */
    0x412e848000000000ull, /* fl64(1e6) */
    0x416312d000000000ull, /* fl64(1e7) */
    0x4197d78400000000ull, /* fl64(1e8) */
    0x41cdcd6500000000ull, /* fl64(1e9) */
    0x4202a05f20000000ull, /* fl64(1e10) */
    0x42374876e8000000ull, /* fl64(1e11) */
    0x426d1a94a2000000ull, /* fl64(1e12) */
    0x42a2309ce5400000ull, /* fl64(1e13) */
    0x42d6bcc41e900000ull, /* fl64(1e14) */
    0x430c6bf526340000ull, /* fl64(1e15) */
    0x4341c37937e08000ull, /* fl64(1e16) */
    0x4376345785d8a000ull, /* fl64(1e17) */
    0x43abc16d674ec800ull, /* fl64(1e18) */
    0x43e158e460913d00ull, /* fl64(1e19) */
    0x4415af1d78b58c40ull, /* fl64(1e20) */
    0x444b1ae4d6e2ef50ull, /* fl64(1e21) */
    0x4480f0cf064dd592ull, /* fl64(1e22) */
};

FALCON_TABLE_QUAL uint32_t FALCON_P10_F32[26] = {
    0x26901d7du, /* fl32(1e-15) */
    0x283424dcu, /* fl32(1e-14) */
    0x29e12e13u, /* fl32(1e-13) */
    0x2b8cbcccu, /* fl32(1e-12) */
    0x2d2febffu, /* fl32(1e-11) */
    0x2edbe6ffu, /* fl32(1e-10) */
    0x3089705fu, /* fl32(1e-9) */
    0x322bcc77u, /* fl32(1e-8) */
    0x33d6bf95u, /* fl32(1e-7) */
    0x358637bdu, /* fl32(1e-6) */
    0x3727c5acu, /* fl32(1e-5) */
    0x38d1b717u, /* fl32(1e-4) */
    0x3a83126fu, /* fl32(1e-3) */
    0x3c23d70au, /* fl32(1e-2) */
    0x3dcccccdu, /* fl32(1e-1) */
    0x3f800000u, /* fl32(1e0) */
    0x41200000u, /* fl32(1e1) */
    0x42c80000u, /* fl32(1e2) */
    0x447a0000u, /* fl32(1e3) */
    0x461c4000u, /* fl32(1e4) */
    0x47c35000u, /* fl32(1e5) */
    0x49742400u, /* fl32(1e6) */
    0x4b189680u, /* fl32(1e7) */
    0x4cbebc20u, /* fl32(1e8) */
    0x4e6e6b28u, /* fl32(1e9) */
    0x501502f9u, /* fl32(1e10) */
};

FALCON_TABLE_QUAL uint16_t FALCON_P10_F16[13] = {
    0x0000u, /* fl16(1e-8) */
    0x0002u, /* fl16(1e-7) */
    0x0011u, /* fl16(1e-6) */
    0x00a8u, /* fl16(1e-5) */
    0x068eu, /* fl16(1e-4) */
    0x1419u, /* fl16(1e-3) */
    0x211fu, /* fl16(1e-2) */
    0x2e66u, /* fl16(1e-1) */
    0x3c00u, /* fl16(1e0) */
    0x4900u, /* fl16(1e1) */
    0x5640u, /* fl16(1e2) */
    0x63d0u, /* fl16(1e3) */
    0x70e2u, /* fl16(1e4) */
};

