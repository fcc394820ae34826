"""GB300-native convergent cross mapping (kEDM hot path) behind a C ABI.

``edm`` is the ctypes binding of ``libedm.so`` (loaded on first use);
``inputs`` holds the seeded synthetic workloads.
"""
