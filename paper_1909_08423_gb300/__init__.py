"""GB300-native PauliNet VMC hot path.

The compute path is the CUDA library ``libpaulinet.so`` (sources in
``csrc/``); ``binding`` marshals arguments to its C ABI.  Importing the
package does not load the library; ``binding`` does, and fails loudly when the
library is missing.
"""
