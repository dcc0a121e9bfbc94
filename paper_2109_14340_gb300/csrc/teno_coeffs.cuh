// Generated by gen_coeffs.py from the integers of Eq. TENO10_AA
// (arXiv 2109.14340, Sec. 4.2) and the derived twelve-point S6; do not edit.
#pragma once

static __constant__ double TENO_Q6[6][6] = {
    {0x1.1f98c98c98c99p+1, -0x1.3aebaebaebaecp+4, 0x1.0e42e983ed943p+5, -0x1.c9f8478478478p+4, 0x1.81ea76a76a76ap+3, -0x1.03ea53fa94feap+1},
    {0.0, 0x1.75e5895895896p+5, -0x1.51c33bde68913p+7, 0x1.280c7ec7ec7ecp+7, -0x1.ff1c3dc3dc3dcp+5, 0x1.5e87db285d308p+3},
    {0.0, 0.0, 0x1.429a1ff754caap+7, -0x1.281c9473f1e9dp+8, 0x1.076432edd9884p+7, -0x1.716643b990ee6p+4},
    {0.0, 0.0, 0.0, 0x1.1c51d41d41d42p+7, -0x1.0692a42a42a43p+7, 0x1.7ad578022acd5p+4},
    {0.0, 0.0, 0.0, 0.0, 0x1.f9eea0ea0ea0fp+4, -0x1.7a4cef79a244dp+3},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0x1.278502fada585p+0},
};

static __constant__ double TENO_Q8[8][8] = {
    {0x1.1e0fb9723ac5cp+1, -0x1.ce76275864377p+4, 0x1.3bd6b5ce1a074p+6, -0x1.d92f416d318b9p+6, 0x1.a4f1e0740a5b0p+6, -0x1.bdf299ba23e43p+5, 0x1.0519309be3ebbp+4, -0x1.0538bbfc8fc1dp+1},
    {0.0, 0x1.84799cd4a10ddp+6, -0x1.1187ee193bb3fp+9, 0x1.a3c7df02cbccep+9, -0x1.7ca8eb0e3d0b2p+9, 0x1.9998b7170e6b8p+8, -0x1.e5dfbdb489e18p+6, 0x1.eb78155475b90p+3},
    {0.0, 0.0, 0x1.8ce47e3e13263p+9, -0x1.387843e0366dap+11, 0x1.2164521d0e13cp+11, -0x1.3cd3fc997b308p+10, 0x1.7d416f7928766p+8, -0x1.864dc99aa4c46p+5},
    {0.0, 0.0, 0.0, 0x1.f8d4a0bf79011p+10, -0x1.de7de8de29e61p+11, 0x1.0b047eab269a4p+11, -0x1.4687aa33c8fd7p+9, 0x1.52cf456d321b0p+6},
    {0.0, 0.0, 0.0, 0.0, 0x1.d014e0b55bed7p+10, -0x1.08730fdaa66fap+11, 0x1.4947f7e24e645p+9, -0x1.5af18a47ca95dp+6},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0x1.33e00b7819f9dp+9, -0x1.86fd6316465aep+8, 0x1.a33a69bfff89cp+5},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0x1.face411eb3c26p+5, -0x1.151dba435a034p+4},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0x1.35c4d1c2ebfb7p+0},
};

static __constant__ double TENO_Q10[10][10] = {
    {0x1.205e62a51c4dcp+1, -0x1.34449c0ee39e4p+5, 0x1.21d551143dccap+7, -0x1.3aae45cfe3b64p+8, 0x1.b321edafebdf9p+8, -0x1.8dc7ac2612257p+8, 0x1.e169d0828747cp+7, -0x1.7461021bbb56bp+6, 0x1.4e82daaa89034p+4, -0x1.0a2fd8e52303fp+1},
    {0.0, 0x1.50f2c2834c23ap+7, -0x1.42f2d4bde706ep+10, 0x1.647d51483fc5fp+11, -0x1.f4057ab7ce1efp+11, 0x1.cec50834f08f6p+11, -0x1.1b10ad5c7bb76p+11, 0x1.ba18c26e018fdp+9, -0x1.908a9eff1eb54p+7, 0x1.413635284aed5p+4},
    {0.0, 0.0, 0x1.3b3b01ef2b67cp+11, -0x1.61cf2a529f7a5p+13, 0x1.f7a9ba3c04d3cp+13, -0x1.d83f67efab794p+13, 0x1.242ecd7dc743ep+13, -0x1.ccf500ad4b3a1p+11, 0x1.a5617cd069304p+9, -0x1.54a45eaf596cfp+6},
    {0.0, 0.0, 0.0, 0x1.93972223766d6p+13, -0x1.239f7eb5703e5p+15, 0x1.152d651a315cap+15, -0x1.5b291bae65a6cp+14, 0x1.14cc344982dcap+13, -0x1.fee49cec12decp+10, 0x1.a080417a07c1ap+7},
    {0.0, 0.0, 0.0, 0.0, 0x1.abb9a4121ad41p+14, -0x1.9c3f317c16178p+15, 0x1.05773783ff781p+15, -0x1.a5b937db11111p+13, 0x1.892a0c14aa3c5p+11, -0x1.436c76ff404b8p+8},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0x1.92d5bb077a4b7p+14, -0x1.02d9bafc5d041p+15, 0x1.a68c2160fa72fp+13, -0x1.8e3b72667fe21p+11, 0x1.4ac9faec6747ap+8},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0x1.50ff7c3610af3p+13, -0x1.167bfc37a5217p+13, 0x1.097f94640eed3p+11, -0x1.bdb95dfc3b77cp+7},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0x1.d20069fe93b66p+10, -0x1.c1a3c482b9536p+9, 0x1.7dbb1cb4db676p+6},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0x1.b732f5137a17cp+6, -0x1.796c631b4bbe5p+4},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0x1.488eb1c659b24p+0},
};

static __constant__ double TENO_Q12[12][12] = {
    {0x1.269b002226085p+1, -0x1.87a6ebf569ab5p+5, 0x1.d56ff0e99f1cfp+7, -0x1.4edaeb3101d00p+9, 0x1.3bf72076f932dp+10, -0x1.9e49857aebad0p+10, 0x1.8155ee8e00e93p+10, -0x1.fcd6c10bcba77p+9, 0x1.d3c7eb488aecap+8, -0x1.1d576bb487155p+7, 0x1.a01384378ed8ep+4, -0x1.12e12b8506f68p+1},
    {0.0, 0x1.08181d212c45dp+8, -0x1.40ad4c0f0349fp+11, 0x1.cede514ca1917p+12, -0x1.b96327ff11f2ep+13, 0x1.2423146b8c802p+14, -0x1.1213a38889d97p+14, 0x1.6cc7f1645ffd6p+13, -0x1.51c8cf63bc13fp+12, 0x1.9edf08f6e0eebp+10, -0x1.30645f19215c3p+8, 0x1.949baf949c8b8p+4},
    {0.0, 0.0, 0x1.8a35c22e445d5p+12, -0x1.1fccd3d5d078dp+15, 0x1.1561704a3d5cdp+16, -0x1.72c68ec555baap+16, 0x1.5ef8222f050a8p+16, -0x1.d6f1703b8fb13p+15, 0x1.b75c554c73431p+14, -0x1.0fadf6ec31a86p+13, 0x1.9138cc8dc9922p+10, -0x1.0c42619f35389p+7},
    {0.0, 0.0, 0.0, 0x1.a8f02cd49e1cdp+15, -0x1.9de9e2d8e4bd4p+17, 0x1.1764a5a1f79a7p+18, -0x1.0ae728db936c2p+18, 0x1.692bf0944b40fp+17, -0x1.53918142d53a2p+16, 0x1.a6f144cd1152bp+14, -0x1.3a5bcd5bf2667p+12, 0x1.a6ec2cd45555dp+8},
    {0.0, 0.0, 0.0, 0.0, 0x1.975e2c5c5b100p+17, -0x1.15b6609365994p+19, 0x1.0bc88ad843239p+19, -0x1.6d855f41691d8p+18, 0x1.5a6c2c5117f98p+17, -0x1.b2ac268aa9ed2p+15, 0x1.45460c653fa92p+13, -0x1.b857cb524b30dp+9},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0x1.7e591edc6e8a9p+18, -0x1.74253217bdda1p+19, 0x1.003e8ad46f9d3p+19, -0x1.e9bda5471ed79p+17, 0x1.359c023c2e362p+16, -0x1.d2a5f68e3472ep+13, 0x1.3dea0ba010df9p+10},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0x1.6d91a1ec7badfp+18, -0x1.fbee568029bf6p+18, 0x1.e980194e99305p+17, -0x1.37e9ec8c9e2d3p+16, 0x1.d994e8b03ddeep+13, -0x1.44d309b2650b7p+10},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0x1.63facc611fb29p+17, -0x1.59fe7e20d7674p+17, 0x1.bc8782880d92fp+15, -0x1.540c0816de8f1p+13, 0x1.d5c894c842a1fp+9},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0x1.5322e0ee98863p+15, -0x1.b74f6eb66a31ep+14, 0x1.52b53235c24ccp+12, -0x1.d76bd92454c47p+8},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0x1.1ee0a31cb1b91p+12, -0x1.bdefef3332b14p+10, 0x1.38c1299fc8dbdp+7},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0x1.5d6c84d459357p+7, -0x1.ee1ef135b705ep+4},
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0x1.60520f198feddp+0},
};

// Linear scheme of the twelve-point candidate S6 at face i+1/2, offsets
// -5..6 (Sec. 4.1 recipe with nu = 7, accuracy constraint 10, 11th-
// difference part 1/200 on cell i).
static __constant__ double TENO_LIN6[12] = {
    -0x1.18c591608ba4ep-11, 0x1.714ca8699bc8dp-8, -0x1.cc2d4b3d96aacp-6, 0x1.76ee011841e20p-4, -0x1.e86f451607ff3p-3, 0x1.58688ba642e5ap-1, 0x1.5349d35457608p-1, -0x1.d9ce5b0767153p-3, 0x1.684d1709a0f7fp-4, -0x1.b8ac132a1572bp-6, 0x1.61b21526ce026p-8, -0x1.0d6c6c18b02bdp-11};

static __constant__ double TENO_DK[3] = {0.5065006634, 0.3699651429, 0.1235341937};
// Renormalised fallback weights w_k = d_k delta_k / sum_j d_j delta_j (double
// division), by (delta_0, delta_1, delta_2) = bits 0..2 of the row index;
// NaN (0/0) when no candidate is kept.
static __constant__ double TENO_FBW[8][3] = {
    {__builtin_nan(""), __builtin_nan(""), __builtin_nan("")},
    {0x1.0000000000000p+0, 0.0, 0.0},
    {0.0, 0x1.0000000000000p+0, 0.0},
    {0x1.27e12c8784fa3p-1, 0x1.b03da6f0f60bcp-2, 0.0},
    {0.0, 0.0, 0x1.0000000000000p+0},
    {0x1.9b9c08ef7a434p-1, 0.0, 0x1.918fdc4216f32p-3},
    {0.0, 0x1.7fd5acb02e066p-1, 0x1.0054a69fa3f33p-2},
    {0x1.03540e11691dbp-1, 0x1.7ad82475a9702p-2, 0x1.f9fefd9e1152cp-4},
};
// Fallback as one linear scheme on offsets -2..2, by (delta_0, delta_1,
// delta_2) = bits 0..2 of the row index.
static __constant__ double TENO_FBK[8][5] = {
    {__builtin_nan(""), __builtin_nan(""), __builtin_nan(""), __builtin_nan(""), __builtin_nan("")},
    {0.0, -0x1.5555555555555p-3, 0x1.aaaaaaaaaaaabp-1, 0x1.5555555555555p-2, 0.0},
    {0.0, 0.0, 0x1.5555555555555p-2, 0x1.aaaaaaaaaaaabp-1, -0x1.5555555555555p-3},
    {0.0, -0x1.8a8190b4b14d9p-4, 0x1.3e9b40ee6d27dp-1, 0x1.16ba1466e82dbp-1, -0x1.202919f5f95d3p-4},
    {0x1.5555555555555p-2, -0x1.2aaaaaaaaaaabp+0, 0x1.d555555555555p+0, 0.0, 0.0},
    {0x1.0bb53d8164a21p-4, -0x1.737298cbb6244p-2, 0x1.078750dd9833bp+0, 0x1.126805f4fc2cdp-2, 0.0},
    {0x1.55c6337f85444p-4, -0x1.2b0d6d0f949bbp-2, 0x1.6aea27a265a10p-1, 0x1.3fdcba92d1055p-1, -0x1.ffc790eae8088p-4},
    {0x1.5154a9140b8c8p-5, -0x1.d40cc7fd25840p-3, 0x1.8b34814102790p-1, 0x1.e896d26da89bdp-2, -0x1.f920309ce1eadp-5},
};

// TENO_SOS6: sum-of-squares form of the large stencil's indicator, variables at offsets [3, 2, 1, -1, -2]
static __constant__ float TENO_SOS6_L[5][5] = {
    {0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {-0x1.47b5f20000000p+2f, 0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f},
    {0x1.482c380000000p+3f, -0x1.dafea20000000p+1f, 0x1.0000000000000p+0f, 0.0f, 0.0f},
    {0x1.2fa78e0000000p+2f, -0x1.70a7380000000p+1f, 0x1.99dd8e0000000p+0f, 0x1.0000000000000p+0f, 0.0f},
    {-0x1.c2506e0000000p-1f, 0x1.3a50a00000000p-1f, -0x1.8c25b20000000p-2f, -0x1.496ec20000000p-2f, 0x1.0000000000000p+0f},
};
static __constant__ float TENO_SOS6_D[5] = {0x1.2785020000000p+0f, 0x1.5a97ca0000000p+0f, 0x1.0daac60000000p+1f, 0x1.07ad2c0000000p+2f, 0x1.a182be0000000p-4f};
static __constant__ float TENO_SOS6_DC[5] = {0x1.9656ea0000000p+4f, 0x1.63784e0000000p+3f, 0x1.92de820000000p+2f, 0x1.5c811a0000000p+2f, 0x1.a182c60000000p-4f};
#define TENO_SOS6_TAU2 0x1.8000060000000p-19f
#define TENO_SOS6_K0 0x1.833f7e0000000p-30f

// TENO_SOS8: sum-of-squares form of the large stencil's indicator, variables at offsets [4, 3, 2, 1, -1, -2, -3]
static __constant__ float TENO_SOS8_L[7][7] = {
    {0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {-0x1.ca07b60000000p+2f, 0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {0x1.5a75ae0000000p+4f, -0x1.736cd00000000p+2f, 0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {-0x1.1eb8d60000000p+5f, 0x1.b842f40000000p+3f, -0x1.1278920000000p+2f, 0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f},
    {-0x1.428e540000000p+4f, 0x1.759f800000000p+3f, -0x1.7814740000000p+2f, 0x1.7524f20000000p+1f, 0x1.0000000000000p+0f, 0.0f, 0.0f},
    {0x1.9629460000000p+2f, -0x1.0cfbe80000000p+2f, 0x1.3113c60000000p+1f, -0x1.5d96960000000p+0f, -0x1.3d4f600000000p-1f, 0x1.0000000000000p+0f, 0.0f},
    {-0x1.afc24c0000000p-1f, 0x1.3f1f580000000p-1f, -0x1.89847a0000000p-2f, 0x1.f0e9e00000000p-3f, 0x1.0a52620000000p-3f, -0x1.75016c0000000p-2f, 0x1.0000000000000p+0f},
};
static __constant__ float TENO_SOS8_D[7] = {0x1.35c4d20000000p+0f, 0x1.5fd7100000000p+0f, 0x1.0c156e0000000p+1f, 0x1.aaffde0000000p+1f, 0x1.bf5b820000000p+3f, 0x1.3d160a0000000p-1f, 0x1.08fdf80000000p-6f};
static __constant__ float TENO_SOS8_DC[7] = {0x1.c2220a0000000p+6f, 0x1.9783a00000000p+5f, 0x1.d2e30e0000000p+4f, 0x1.26cfb40000000p+4f, 0x1.8763da0000000p+4f, 0x1.b096ca0000000p-1f, 0x1.08fdfe0000000p-6f};
#define TENO_SOS8_TAU2 0x1.8000060000000p-19f
#define TENO_SOS8_K0 0x1.cea02c0000000p-26f

// TENO_SOS10: sum-of-squares form of the large stencil's indicator, variables at offsets [5, 4, 3, 2, 1, -1, -2, -3, -4]
static __constant__ float TENO_SOS10_L[9][9] = {
    {0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {-0x1.26131a0000000p+3f, 0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {0x1.296e4e0000000p+5f, -0x1.f938960000000p+2f, 0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {-0x1.5b4ac20000000p+6f, 0x1.ae9ebe0000000p+4f, -0x1.9808cc0000000p+2f, 0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {0x1.01bd200000000p+7f, -0x1.9df0960000000p+5f, 0x1.11f7d60000000p+4f, -0x1.37b8d20000000p+2f, 0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {0x1.4485c00000000p+6f, -0x1.700fac0000000p+5f, 0x1.5d85b00000000p+4f, -0x1.4683f00000000p+3f, 0x1.2490320000000p+2f, 0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f},
    {-0x1.096a7a0000000p+5f, 0x1.552ab60000000p+4f, -0x1.686ef60000000p+3f, 0x1.7f99800000000p+2f, -0x1.919ae40000000p+1f, -0x1.d0ae740000000p-1f, 0x1.0000000000000p+0f, 0.0f, 0.0f},
    {0x1.f48d960000000p+2f, -0x1.65f7140000000p+2f, 0x1.9964be0000000p+1f, -0x1.df1c040000000p+0f, 0x1.16e5f20000000p+0f, 0x1.7eb3ae0000000p-2f, -0x1.721bea0000000p-1f, 0x1.0000000000000p+0f, 0.0f},
    {-0x1.9ece6c0000000p-1f, 0x1.45f4de0000000p-1f, -0x1.8bda940000000p-2f, 0x1.f1e6ba0000000p-3f, -0x1.391e760000000p-3f, -0x1.e330000000000p-5f, 0x1.37eb040000000p-3f, -0x1.7996100000000p-2f, 0x1.0000000000000p+0f},
};
static __constant__ float TENO_SOS10_D[9] = {0x1.488eb20000000p+0f, 0x1.6914c40000000p+0f, 0x1.0911840000000p+1f, 0x1.a769b20000000p+1f, 0x1.512df40000000p+2f, 0x1.36f7de0000000p+5f, 0x1.3605d40000000p+1f, 0x1.f7c9680000000p-4f, 0x1.4bb6900000000p-9f};
static __constant__ float TENO_SOS10_DC[9] = {0x1.ef67300000000p+8f, 0x1.c67c1e0000000p+7f, 0x1.fae0f80000000p+6f, 0x1.3ff9f60000000p+6f, 0x1.a36aae0000000p+5f, 0x1.6be1040000000p+6f, 0x1.22ac5a0000000p+2f, 0x1.58c6980000000p-3f, 0x1.4bb6960000000p-9f};
#define TENO_SOS10_TAU2 0x1.8000060000000p-19f
#define TENO_SOS10_K0 0x1.0b2d620000000p-21f

// TENO_SOS12: sum-of-squares form of the large stencil's indicator, variables at offsets [6, 5, 4, 3, 2, 1, -1, -2, -3, -4, -5]
static __constant__ float TENO_SOS12_L[11][11] = {
    {0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {-0x1.6708a00000000p+3f, 0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {0x1.c680760000000p+5f, -0x1.3f72a00000000p+3f, 0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {-0x1.568a380000000p+7f, 0x1.636ac00000000p+5f, -0x1.0ecbe20000000p+3f, 0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {0x1.5559920000000p+8f, -0x1.d02d4a0000000p+6f, 0x1.f704600000000p+4f, -0x1.bd54320000000p+2f, 0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {-0x1.d80abe0000000p+8f, 0x1.89fde20000000p+7f, -0x1.0d3dba0000000p+6f, 0x1.4e31920000000p+4f, -0x1.5ce6080000000p+2f, 0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {-0x1.3ff5420000000p+8f, 0x1.68701e0000000p+7f, -0x1.48c2b20000000p+6f, 0x1.28a8f00000000p+5f, -0x1.007e6e0000000p+4f, 0x1.a453bc0000000p+2f, 0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f, 0.0f},
    {0x1.334cda0000000p+7f, -0x1.84df9a0000000p+6f, 0x1.85b6520000000p+5f, -0x1.8ab71e0000000p+4f, 0x1.86b4420000000p+3f, -0x1.79aee20000000p+2f, -0x1.30e5100000000p+0f, 0x1.0000000000000p+0f, 0.0f, 0.0f, 0.0f},
    {-0x1.85d7200000000p+5f, 0x1.1131180000000p+5f, -0x1.268a2c0000000p+4f, 0x1.46296c0000000p+3f, -0x1.649bb00000000p+2f, 0x1.8258900000000p+1f, 0x1.7396be0000000p-1f, -0x1.13be7c0000000p+0f, 0x1.0000000000000p+0f, 0.0f, 0.0f},
    {0x1.25fe240000000p+3f, -0x1.c3bf580000000p+2f, 0x1.01ded20000000p+2f, -0x1.3283700000000p+1f, 0x1.69a1b00000000p+0f, -0x1.aa016e0000000p-1f, -0x1.cede200000000p-3f, 0x1.cd36220000000p-2f, -0x1.7a30b00000000p-1f, 0x1.0000000000000p+0f, 0.0f},
    {-0x1.8f76080000000p-1f, 0x1.4e11300000000p-1f, -0x1.8eed1e0000000p-2f, 0x1.f6360c0000000p-3f, -0x1.3a94520000000p-3f, 0x1.8b26ba0000000p-4f, 0x1.d612920000000p-6f, -0x1.1abfb80000000p-4f, 0x1.383d240000000p-3f, -0x1.797ae60000000p-2f, 0x1.0000000000000p+0f},
};
static __constant__ float TENO_SOS12_D[11] = {0x1.6052100000000p+0f, 0x1.76c0280000000p+0f, 0x1.0629300000000p+1f, 0x1.a35f0e0000000p+1f, 0x1.4de26c0000000p+2f, 0x1.0a01540000000p+3f, 0x1.8049fc0000000p+6f, 0x1.e97b8a0000000p+2f, 0x1.223d9e0000000p-1f, 0x1.8943600000000p-6f, 0x1.9303c20000000p-12f};
static __constant__ float TENO_SOS12_DC[11] = {0x1.10d7920000000p+11f, 0x1.f762e60000000p+9f, 0x1.0c3f360000000p+9f, 0x1.52df260000000p+8f, 0x1.b473800000000p+7f, 0x1.218ae80000000p+7f, 0x1.30b05e0000000p+8f, 0x1.3dbe160000000p+4f, 0x1.1270660000000p+0f, 0x1.0d1dd60000000p-5f, 0x1.9303ca0000000p-12f};
#define TENO_SOS12_TAU2 0x1.8000060000000p-19f
#define TENO_SOS12_K0 0x1.309c9e0000000p-17f

