"""GB300-native two-stage compact gas-kinetic scheme on tetrahedral meshes.

``gks``     ctypes binding of libgks (the C ABI in include/gks.h)
``inputs``  seeded synthetic meshes, initial fields and exact solutions
``_build``  in-tree build of libgks.so for sm_103a
"""
