"""GB300-native blocked Floyd-Warshall all-pairs shortest paths.

The compute path is the C-ABI library ``libapsp.so`` built from ``csrc/`` for
sm_103a; ``binding`` marshals arguments to it.  Importing this package does not
load the library: ``binding.lib()`` does, and raises if it has not been built.
"""
