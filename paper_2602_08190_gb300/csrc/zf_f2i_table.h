// zf_f2i_table.h -- written by gen_f2i_table.py (exact integer arithmetic); do not edit.
// Row e (1..18): { ceil(2^(64+s)/5^e), ceil(2^(128+s)/5^e) high word, low word, s = floor(log2 5^e) }.
#pragma once
#define ZF_F2I_RECIP_ROWS \
    {0x0000000000000000ull, 0x0000000000000000ull, 0x0000000000000000ull, 0u}, \
    {0xcccccccccccccccdull, 0xccccccccccccccccull, 0xcccccccccccccccdull, 2u}, \
    {0xa3d70a3d70a3d70bull, 0xa3d70a3d70a3d70aull, 0x3d70a3d70a3d70a4ull, 4u}, \
    {0x83126e978d4fdf3cull, 0x83126e978d4fdf3bull, 0x645a1cac083126eaull, 6u}, \
    {0xd1b71758e219652cull, 0xd1b71758e219652bull, 0xd3c36113404ea4a9ull, 9u}, \
    {0xa7c5ac471b478424ull, 0xa7c5ac471b478423ull, 0x0fcf80dc33721d54ull, 11u}, \
    {0x8637bd05af6c69b6ull, 0x8637bd05af6c69b5ull, 0xa63f9a49c2c1b110ull, 13u}, \
    {0xd6bf94d5e57a42bdull, 0xd6bf94d5e57a42bcull, 0x3d32907604691b4dull, 16u}, \
    {0xabcc77118461cefdull, 0xabcc77118461cefcull, 0xfdc20d2b36ba7c3eull, 18u}, \
    {0x89705f4136b4a598ull, 0x89705f4136b4a597ull, 0x31680a88f8953031ull, 20u}, \
    {0xdbe6fecebdedd5bfull, 0xdbe6fecebdedd5beull, 0xb573440e5a884d1cull, 23u}, \
    {0xafebff0bcb24aaffull, 0xafebff0bcb24aafeull, 0xf78f69a51539d749ull, 25u}, \
    {0x8cbccc096f5088ccull, 0x8cbccc096f5088cbull, 0xf93f87b7442e45d4ull, 27u}, \
    {0xe12e13424bb40e14ull, 0xe12e13424bb40e13ull, 0x2865a5f206b06fbaull, 30u}, \
    {0xb424dc35095cd810ull, 0xb424dc35095cd80full, 0x538484c19ef38c95ull, 32u}, \
    {0x901d7cf73ab0acdaull, 0x901d7cf73ab0acd9ull, 0x0f9d37014bf60a11ull, 34u}, \
    {0xe69594bec44de15cull, 0xe69594bec44de15bull, 0x4c2ebe687989a9b4ull, 37u}, \
    {0xb877aa3236a4b44aull, 0xb877aa3236a4b449ull, 0x09befeb9fad487c3ull, 39u}, \
    {0x9392ee8e921d5d08ull, 0x9392ee8e921d5d07ull, 0x3aff322e62439fd0ull, 41u}
