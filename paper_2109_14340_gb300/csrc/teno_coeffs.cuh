// Generated by gen_coeffs.py from the integers of Eq. TENO10_AA
// (arXiv 2109.14340, Sec. 4.2); do not edit.
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

