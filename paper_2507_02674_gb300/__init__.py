"""GB300-native real-time image-based lighting of glints (Kneiphof & Klein, EGSR 2025).

The compute path is the CUDA library ``libglint.so`` (C ABI declared in
``include/glint.h``); ``paper_2507_02674_gb300.glint`` is its thin ctypes
binding.  ``paper_2507_02674_gb300.synth`` generates seeded inputs.
"""
