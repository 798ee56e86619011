"""Plain CPU reference (oracle) of the world cache and the screen-probe stage.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
baseline leg of bench.py may import this package; the product path (the
CUDA library and its Python binding) never does, and this package imports
nothing from it.

Everything is float64 except the cell key, which the method defines as an
integer function of the float32 hit record (explicit float32 operations,
see key.py), so that keys can be compared bit for bit.

Modules, by the part of the paper they follow:
  hashing.py  -- bucket hash and fingerprint (Section 2.2.1)
  key.py      -- cell descriptor: quantised position, direction, distance LOD
                 (Section 2.2.1) and the light-leak bit (Section 2.2.2);
                 adaptive cell size (Algorithm 6)
  cache.py    -- insert/accumulate, resolve with exponential moving average
                 (Section 2.2.3), decay and eviction (Section 2.2.1), lookup
  hemioct.py  -- hemispherical octahedral 8x8 cell geometry (Section 2.1)
  sh.py       -- 3-band spherical harmonics, cosine-lobe convolution
                 (Section 2.4.2)
  probes.py   -- probe spawn with Halton jitter (Section 2.1.1), probe mask
                 and its MIP chain, directional probe search (Section 2.1.5,
                 Algorithm 3), probe irradiance (Section 2.4.2) and per-pixel
                 interpolation (Section 2.4.1)
  frame.py    -- one frame of the whole path, in the paper's pass order
  surrogate.py -- the learned radiance surrogate (no paper section: multiresolution hash
                 encoding, relative L2 loss and Adam from their own publications)

Parity pins are in tests/test_oracle_*.py; every function here is pinned
there against closed forms, brute force or library routines.
"""
